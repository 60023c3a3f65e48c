// The tile kernel of the split-BF16 product (included by bsmm_split.cu).
//
// Warp roles (12 warps, one CTA per SM):
//   warps 0-7   drain: every DRAIN chunks they read the FP32 accumulator (warp w: TMEM lane
//               quarter w % 4, columns 32 * (w / 4) ..) into double-float (hi, lo) sums in
//               registers, release the accumulator, and write C after a tile's last period;
//   warps 8-10  producers: thread q < 64 copies A rows q and q + 64, thread q >= 64 copies
//               B rows q - 64 and q - 32: per chunk the rows' pieces of the chunk's atoms,
//               three BF16 planes each, with cp.async (zero fill for absent blocks), then
//               marks the stage full;
//   warp 11     lane 0 issues the 18 MMAs of a chunk (3 K steps x 6 split products) into
//               one of two TMEM accumulators and commits them to the stage's "empty"
//               barrier, and at the end of a drain period to the accumulator's "full" barrier.
// Stages rotate over one running chunk counter across all tiles of the CTA; accumulators
// over one running period counter; every wait computes its parity from those counters.
// Producers signal a chunk LAG chunks after issuing it: they wait for their own copies
// (cp.async.wait_group), make them visible to the tensor core (fence.proxy.async) and
// arrive, so LAG + 1 chunks of copies per thread are in flight.
//
// Every wait is bounded (about two seconds) and also ends when another role has given up:
// the CTA then stops issuing work, retires its own copies and MMAs (bounded), frees its
// tensor memory and returns with bit 16 of the context flag set.
constexpr int NS = 4;    // shared-memory stages
constexpr int LAG = 2;   // chunks a producer keeps in flight before signalling
constexpr int N_PROD = (MT + NT) / 2;  // producer threads (two tile rows each)
constexpr int N_DRAIN = 256;           // drain threads
constexpr int W_PROD = 8, W_MMA = 11;  // first producer warp, MMA warp

struct Bars {
    uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], done;
    uint32_t tmem_slot;
    int abort_flag;
};
static_assert(sizeof(Bars) <= BAR_BYTES, "barrier block");
static_assert(NS * STAGE + BAR_BYTES <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ bool bar_try(uint32_t addr, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase; gives up when another role has set the abort flag.
__device__ __forceinline__ bool bar_wait(uint32_t addr, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!bar_try(addr, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Bounded wait that ignores the abort flag (retiring work already issued).
__device__ __forceinline__ bool bar_wait_plain(uint32_t addr, uint32_t parity)
{
    const long long t0 = clock64();
    while (!bar_try(addr, parity))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void bar_arrive(uint32_t addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void bar_commit(uint32_t addr)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(addr)
        : "memory");
}

// block indices of this thread's row for the atoms of chunk c (-1: absent)
template <int NB>
__device__ __forceinline__ void load_index(const SplitArgs &p, int64_t kb, int64_t kn, int c,
                                           int slot, int32_t (&blk)[KLayout<NB>::CA])
{
    constexpr int CA = KLayout<NB>::CA, W = MT / NB + NT / NB;
#pragma unroll
    for (int a = 0; a < CA; ++a) {
        const int64_t kidx = (int64_t)c * CA + a;
        blk[a] = (slot >= 0 && kidx < kn) ? __ldg(&p.table[(kb + kidx) * W + slot]) : -1;
    }
}

// copy this thread's row of one chunk (all atoms, three planes) into a stage
template <int NB>
__device__ __forceinline__ void gather_chunk(const SplitArgs &p, uint32_t stage, bool a_side,
                                             int row, int o,
                                             const int32_t (&blk)[KLayout<NB>::CA])
{
    constexpr int CA = KLayout<NB>::CA, MW = KLayout<NB>::MAINW;
    const uint32_t base = a_side ? stage : stage + 3 * A_PLANE;
    const int plane = a_side ? A_PLANE : B_PLANE;
#pragma unroll
    for (int a = 0; a < CA; ++a) {
        const bool have = blk[a] >= 0;
        const int64_t r = have ? (int64_t)blk[a] * NB + o : 0;
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            const uint32_t d = base + pl * plane;
            if (MW) {
                const __nv_bfloat16 *m = (a_side ? p.sa_main[pl] : p.sb_main[pl]) + r * MW;
                cp16z(d + tile_off(row, KLayout<NB>::main_col(a), 0), m, have ? 16u : 0u);
            }
            const __nv_bfloat16 *tl = (a_side ? p.sa_tail[pl] : p.sb_tail[pl]) + r * TAILW;
            cp8z(d + tile_off(row, KLayout<NB>::tail_col(a), (a & 1) * 8), tl, have ? 8u : 0u);
        }
    }
}

// Epilogue of one drain thread: accumulator row arow = (atom ia of group g, orbital a),
// columns 32*HALF .. +31 = (atom of group h, orbital); each block (ia, j) that P_C holds is
// found by one binary search over row ia of P_C and written as beta*C + alpha*(hi + lo).
template <int NB, int HALF>
__device__ __forceinline__ void write_rows(const SplitArgs &p, int2 tg, int arow,
                                           const float (&hi)[32], const float (&lo)[32])
{
    constexpr int GI = MT / NB, GJ = NT / NB;
    constexpr int J0 = (HALF * 32) / NB, J1 = (HALF * 32 + 31) / NB;
    if (arow >= GI * NB) return;
    const int ia = p.g_atoms[(int64_t)tg.x * GI + arow / NB];
    if (ia < 0) return;
    const int a = arow % NB;
    const int64_t r0 = p.c_rp[ia], r1 = p.c_rp[ia + 1];
#pragma unroll
    for (int jl = J0; jl <= J1; ++jl) {
        if (jl >= GJ) continue;
        const int j = p.h_atoms[(int64_t)tg.y * GJ + jl];
        if (j < 0) continue;
        int64_t lo_i = r0, hi_i = r1;
        while (lo_i < hi_i) {
            const int64_t mid = (lo_i + hi_i) >> 1;
            if (p.c_col[mid] < j)
                lo_i = mid + 1;
            else
                hi_i = mid;
        }
        if (lo_i >= r1 || p.c_col[lo_i] != j) continue;
        double *dst = p.C + lo_i * p.c_stride + a * NB;
#pragma unroll
        for (int bo = 0; bo < NB; ++bo) {
            const int x = jl * NB + bo - HALF * 32;
            if (x < 0 || x >= 32) continue;
            const double v = (double)hi[x] + (double)lo[x];
            dst[bo] = p.beta == 0.0 ? p.alpha * v : p.beta * dst[bo] + p.alpha * v;
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(ST, 1) k_bsmm_split(const SplitArgs p)
{
    constexpr int GI = MT / NB, GJ = NT / NB, CA = KLayout<NB>::CA;
    extern __shared__ __align__(1024) uint8_t smem[];
    Bars *bars = reinterpret_cast<Bars *>(smem + NS * STAGE);
    volatile int *abort_flag = &bars->abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t sm0 = smem_u32(smem);

    for (int e = t; e < NS * STAGE / 16; e += ST)
        reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->full[s])),
                         "r"(N_PROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->empty[s])),
                         "r"(1));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                             smem_u32(&bars->acc_full[b])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                             smem_u32(&bars->acc_empty[b])),
                         "r"(N_DRAIN));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->done)), "r"(1));
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = bars->tmem_slot;

    if (warp >= W_PROD && warp < W_MMA) {
        // ------------------------------------------------------------ producers
        const int q = t - W_PROD * 32;
        const bool a_side = q < MT / 2;
        int row[2], slot[2], o[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            row[rr] = a_side ? q + rr * (MT / 2) : q - MT / 2 + rr * (NT / 2);
            slot[rr] = -1;
            if (a_side && row[rr] < GI * NB) slot[rr] = row[rr] / NB;
            if (!a_side && row[rr] < GJ * NB) slot[rr] = GI + row[rr] / NB;
            o[rr] = row[rr] % NB;
        }
        uint32_t cg = 0;  // running chunk counter
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t kb = p.kstart[tile], kn = p.kstart[tile + 1] - kb;
            const int nch = (int)((kn + CA - 1) / CA);
            int32_t nxt[2][CA];
            if (nch > 0)
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) load_index<NB>(p, kb, kn, 0, slot[rr], nxt[rr]);
            for (int c = 0; c < nch; ++c, ++cg) {
                const int s = (int)(cg % NS);
                if (cg >= (uint32_t)NS &&
                    !bar_wait(smem_u32(&bars->empty[s]), ((cg / NS) + 1) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                int32_t cur[2][CA];
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                    for (int a = 0; a < CA; ++a) cur[rr][a] = nxt[rr][a];
                if (c + 1 < nch)
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr)
                        load_index<NB>(p, kb, kn, c + 1, slot[rr], nxt[rr]);
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
                    gather_chunk<NB>(p, sm0 + s * STAGE, a_side, row[rr], o[rr], cur[rr]);
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (cg >= (uint32_t)LAG) {
                    asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_arrive(smem_u32(&bars->full[(cg - LAG) % NS]));
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (ok) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (uint32_t q = cg > (uint32_t)LAG ? cg - LAG : 0u; q < cg; ++q)
                bar_arrive(smem_u32(&bars->full[q % NS]));
        }
    } else if (warp == W_MMA) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            uint32_t cg = 0, pg = 0;
            bool ok = true, issued = false;
            const int pq[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
            for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
                const int64_t kn = p.kstart[tile + 1] - p.kstart[tile];
                const int nch = (int)((kn + CA - 1) / CA);
                for (int c = 0; c < nch; ++c, ++cg) {
                    const uint32_t b = pg & 1u;
                    if (c % DRAIN == 0 && pg >= 2 &&
                        !bar_wait(smem_u32(&bars->acc_empty[b]), ((pg / 2) + 1) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int s = (int)(cg % NS);
                    if (!bar_wait(smem_u32(&bars->full[s]), (cg / NS) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ab = sm0 + s * STAGE, bb = ab + 3 * A_PLANE;
                    const uint32_t acc_addr = tmem + b * NT;
#pragma unroll
                    for (int ks = 0; ks < KSTEPS; ++ks)
#pragma unroll
                        for (int x = 0; x < 6; ++x) {
                            const uint64_t ad = smem_desc(ab + pq[x][0] * A_PLANE + ks * 256);
                            const uint64_t bd = smem_desc(bb + pq[x][1] * B_PLANE + ks * 256);
                            const uint32_t acc = (c % DRAIN == 0 && ks == 0 && x == 0) ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                    acc_addr),
                                "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                        }
                    bar_commit(smem_u32(&bars->empty[s]));
                    issued = true;
                    if (c % DRAIN == DRAIN - 1 || c == nch - 1) {
                        bar_commit(smem_u32(&bars->acc_full[b]));
                        ++pg;
                    }
                }
            }
            if (issued) {  // retire every MMA before the tensor memory is released
                bar_commit(smem_u32(&bars->done));
                if (!bar_wait_plain(smem_u32(&bars->done), 0u)) *abort_flag = 1;
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ drain and epilogue
        const int quarter = warp & 3, half = warp >> 2;
        const int arow = quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
        uint32_t pg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int2 tg = p.tiles[tile];
            const int64_t kn = p.kstart[tile + 1] - p.kstart[tile];
            const int nch = (int)((kn + CA - 1) / CA);
            const int np = (nch + DRAIN - 1) / DRAIN;
            float hi[32], lo[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) hi[x] = lo[x] = 0.f;
            for (int d = 0; d < np; ++d, ++pg) {
                const uint32_t b = pg & 1u;
                if (!bar_wait(smem_u32(&bars->acc_full[b]), (pg / 2) & 1u, abort_flag)) {
                    ok = false;
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
                        : "r"(lane_addr + b * NT + q * 16));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int x = 0; x < 16; ++x)
                        two_sum_add(hi[q * 16 + x], lo[q * 16 + x], __uint_as_float(v[x]));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                bar_arrive(smem_u32(&bars->acc_empty[b]));
            }
            if (!ok) break;
            if (half == 0)
                write_rows<NB, 0>(p, tg, arow, hi, lo);
            else
                write_rows<NB, 1>(p, tg, arow, hi, lo);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (t == 0 && *abort_flag) atomicOr(p.flag, 16);
    if (warp == W_MMA) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
}
