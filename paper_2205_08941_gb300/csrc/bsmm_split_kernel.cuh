// The tile kernel of the split-BF16 product (included by bsmm_split.cu).
//
// Roles: threads 0..127 gather the 128 A rows of a chunk, threads 128..191 the 64 B rows
// (16-byte cp.async pieces, block indices from the tile's index table, zeros for absent
// blocks); thread 0 issues the 24 MMAs of a chunk (4 K steps x 6 split products) and
// commits them to the chunk's stage barrier; all 8 warps drain the accumulator (warps w and
// w+4 read TMEM lane quarter w, columns 0..31 and 32..63).
//
// Pipeline: NS shared stages.  Chunk c lives in stage c % NS.  Gathers run NS-1 chunks
// ahead of the tensor core (cp.async groups, one per chunk); a stage is refilled only
// after the barrier of the MMAs that last read it has completed.
constexpr int NS = 3;

// block indices of this thread's row for the four atoms of chunk c (-1: absent)
template <int NB>
__device__ __forceinline__ void load_index(const SplitArgs &p, int64_t kb, int64_t kn, int c,
                                           int slot, int32_t blk[4])
{
    constexpr int GI = MT / NB, GJ = NT / NB, W = GI + GJ;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int64_t kidx = (int64_t)c * 4 + kk;
        blk[kk] = (slot >= 0 && kidx < kn) ? p.table[(kb + kidx) * W + slot] : -1;
    }
}

template <int NB>
__device__ __forceinline__ void gather_chunk(const SplitArgs &p, uint8_t *stg, uint32_t sbase,
                                             const int32_t blk[4], bool a_role, bool b_role,
                                             int grow, int o)
{
    if (!(a_role || b_role)) return;
    const uint32_t dbase = a_role ? sbase : sbase + 3 * A_PLANE;
    uint8_t *gbase = a_role ? stg : stg + 3 * A_PLANE;
    const int plane = a_role ? A_PLANE : B_PLANE;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            const uint32_t d = dbase + pl * plane;
            if (blk[kk] >= 0) {
                const __nv_bfloat16 *src =
                    (a_role ? p.sa[pl] : p.sb[pl]) + ((int64_t)blk[kk] * NB + o) * KP;
                cp16(d + cm_off(grow, 2 * kk), src);
                cp16(d + cm_off(grow, 2 * kk + 1), src + 8);
            } else {
                uint8_t *g = gbase + pl * plane;
                *reinterpret_cast<uint4 *>(g + cm_off(grow, 2 * kk)) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(g + cm_off(grow, 2 * kk + 1)) =
                    make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(ST, 1) k_bsmm_split(const SplitArgs p)
{
    constexpr int GI = MT / NB, GJ = NT / NB;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + NS * STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + NS * STAGE + 8 * NS);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const bool a_role = t < MT, b_role = t >= MT && t < MT + NT;
    const int grow = a_role ? t : t - MT;
    const int arow = (warp & 3) * 32 + lane, half = warp >> 2;

    for (int e = t; e < NS * STAGE / 16; e += ST)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (t == 0) {
        for (int s = 0; s < NS; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[s])),
                         "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * 32);
    const uint32_t sm0 = smem_u32(smem);

    uint32_t phase[NS];
    bool pending[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        phase[s] = 0u;
        pending[s] = false;
    }
    bool failed = false;

    // wait (CTA-uniformly, bounded) until the MMAs that last read stage s are complete
    auto free_stage = [&](int s) -> bool {
        if (!pending[s]) return true;
        const bool ok = mbar_wait(smem_u32(&mbar[s]), phase[s]);
        if (__syncthreads_or(!ok)) return false;
        phase[s] ^= 1u;
        pending[s] = false;
        return true;
    };

    for (int tile = blockIdx.x; tile < p.n_tiles && !failed; tile += gridDim.x) {
        const int2 tg = p.tiles[tile];
        const int64_t kb = p.kstart[tile], kn = p.kstart[tile + 1] - kb;
        int slot = -1;
        if (a_role && grow < GI * NB) slot = grow / NB;
        if (b_role && grow < GJ * NB) slot = GI + grow / NB;
        const int o = grow % NB;
        float hi[32], lo[32];
#pragma unroll
        for (int x = 0; x < 32; ++x) hi[x] = lo[x] = 0.f;
        const int nch = (int)((kn + 3) / 4);
        // prologue: the first NS-1 chunks; nxt holds the indices of the next chunk to gather,
        // loaded one iteration ahead so the gather waits for one memory round trip only
        int32_t nxt[4];
        for (int c = 0; c < NS - 1 && c < nch; ++c) {
            if (!free_stage(c % NS)) {
                failed = true;
                break;
            }
            load_index<NB>(p, kb, kn, c, slot, nxt);
            gather_chunk<NB>(p, smem + (c % NS) * STAGE, sm0 + (c % NS) * STAGE, nxt, a_role,
                             b_role, grow, o);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        load_index<NB>(p, kb, kn, NS - 1, slot, nxt);
        for (int c = 0; c < nch && !failed; ++c) {
            const int s = c % NS;
            if (c + 1 < nch)
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            else
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ab = sm0 + s * STAGE, bbase = ab + 3 * A_PLANE;
                const int pq[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
#pragma unroll
                for (int ks = 0; ks < KCH / 16; ++ks)
#pragma unroll
                    for (int x = 0; x < 6; ++x) {
                        const uint64_t ad = smem_desc(ab + pq[x][0] * A_PLANE + ks * 256);
                        const uint64_t bd = smem_desc(bbase + pq[x][1] * B_PLANE + ks * 256);
                        const uint32_t acc = (c % DRAIN == 0 && ks == 0 && x == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                tmem),
                            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                    }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&mbar[s]))
                    : "memory");
            }
            pending[s] = true;
            // refill: chunk c + NS - 1 goes to the stage chunk c - 1 used
            const int cn = c + NS - 1;
            if (cn < nch) {
                if (!free_stage(cn % NS)) {
                    failed = true;
                    break;
                }
                gather_chunk<NB>(p, smem + (cn % NS) * STAGE, sm0 + (cn % NS) * STAGE, nxt,
                                 a_role, b_role, grow, o);
                asm volatile("cp.async.commit_group;" ::: "memory");
                load_index<NB>(p, kb, kn, cn + 1, slot, nxt);
            }
            if (c % DRAIN == DRAIN - 1 || c == nch - 1) {
                if (!free_stage(s)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    uint32_t v[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"
                        "%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                          "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]),
                          "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr + q * 16));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int x = 0; x < 16; ++x)
                        two_sum_add(hi[q * 16 + x], lo[q * 16 + x], __uint_as_float(v[x]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (failed) break;
        // epilogue: accumulator row arow = (atom ia, orbital a), columns 32*half .. +31 =
        // (atom of group h, orbital) of every block P_C holds
        const int ia = arow < GI * NB ? p.g_atoms[(int64_t)tg.x * GI + arow / NB] : -1;
        if (ia >= 0) {
            const int a = arow % NB;
            int cached_jl = -1;
            double *dst = nullptr;
#pragma unroll
            for (int x = 0; x < 32; ++x) {
                const int col = half * 32 + x;
                const int jl = col / NB, bo = col % NB;
                if (jl >= GJ) continue;
                if (jl != cached_jl) {
                    cached_jl = jl;
                    dst = nullptr;
                    const int j = p.h_atoms[(int64_t)tg.y * GJ + jl];
                    if (j >= 0) {
                        int64_t lo_i = p.c_rp[ia], hi_i = p.c_rp[ia + 1];
                        while (lo_i < hi_i) {
                            const int64_t mid = (lo_i + hi_i) >> 1;
                            if (p.c_col[mid] < j)
                                lo_i = mid + 1;
                            else
                                hi_i = mid;
                        }
                        if (lo_i < p.c_rp[ia + 1] && p.c_col[lo_i] == j)
                            dst = p.C + lo_i * p.c_stride + a * NB;
                    }
                }
                if (!dst) continue;
                const double v = (double)hi[x] + (double)lo[x];
                dst[bo] = p.beta == 0.0 ? p.alpha * v : p.beta * dst[bo] + p.alpha * v;
            }
        }
    }
    if (failed && t == 0) atomicOr(p.flag, 16);
    // retire outstanding commits before releasing tensor memory
    for (int s = 0; s < NS; ++s)
        if (pending[s]) mbar_wait(smem_u32(&mbar[s]), phase[s]);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
}
