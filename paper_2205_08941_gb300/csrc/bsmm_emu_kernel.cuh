// The tile kernel of the emulated-FP64 product (included by bsmm_split.cu after the split
// kernel, whose barrier, copy and timeout helpers it shares).
//
// Operands are eight BF16 digit planes per value (emu_digits.cuh): A_p, B_q with planes
// pre-scaled by 2^(-8p), so the MMA of planes p and q lands at level p + q.  Per K step the
// MMA thread issues the 36 products with p + q <= 7, level by level, into six FP32 accumulators in tensor
// memory: levels 0 to 4 each alone -- over one scale period a level-l sum is an integer
// times 2^(-8 l) of magnitude at most (l + 1) * 192 * 128^2 < 2^24 (192 K values per
// period), hence exact -- and levels 5-7 together (rounded, but 2^-40 below level 0, so its
// rounding stays near 2^-64 of the group's scale, as does the digit split itself).  A scale
// period is a run of chunks whose K groups share a scale group (four K groups, sixteen
// 9-orbital atoms).  At its end the drain warps scale every level by
// 2^(E_A(row) + E_B(column) - 14) and add it into a three-float sum (h, m, l): h and m in
// tensor memory beside the accumulators, l (the smallest word) in shared memory (column-
// major, so the lanes of a warp, which own consecutive rows, hit distinct banks).  After a
// tile's last period C = beta C + alpha (h + m + l) is written in FP64.
//
// Warp roles (10 warps, one CTA per SM):
//   warp 0      producer: lane 0 copies every K step of every chunk (A: 8 planes x 128 rows
//               x 16 K, 32 KB; B: 8 planes x 64 rows, 16 KB) into a free stage with two TMA
//               bulk copies completing on the stage's "full" barrier;
//   warp 1      lane 0 issues the 36 MMAs of each K step and commits the stage to its
//               "empty" barrier; at a period's end it commits the accumulators to
//               "acc_full" and, before the next period, waits on "acc_empty";
//   warps 2-9   drain (lane quarter w % 4, columns 32 ((w - 2) / 4) ..) and epilogue.
// Tensor memory (512 columns): levels 0-5 at columns 0, 64, ..., 320; h and m at 384 and
// 448.  The accumulators are single-buffered (the sums take the rest), so the MMA thread
// waits while a period drains.
//
// Every wait is bounded as in the split kernel; a CTA that gives up retires its copies and
// MMAs, frees its tensor memory and sets bit 16 of the context flag.
constexpr int NSE = 4;                       // shared-memory stages (one K step each)
constexpr int E_APLANE = MT * 16 * 2;        // 4 KB: one A digit plane of one K step
constexpr int E_BPLANE = NT * 16 * 2;        // 2 KB
constexpr int E_AKSTEP = EMU_P * E_APLANE;   // 32 KB
constexpr int E_BKSTEP = EMU_P * E_BPLANE;   // 16 KB
constexpr int E_APANEL = KSTEPS * E_AKSTEP;  // 96 KB: one packed A panel
constexpr int E_BPANEL = KSTEPS * E_BKSTEP;  // 48 KB
constexpr int E_STAGE = E_AKSTEP + E_BKSTEP;
constexpr int E_SBO = 256;                   // bytes between 8-row groups (2 core columns)
constexpr int E_LEVELS = 6;                  // accumulators: levels 0-4, then 5-7 merged
constexpr int E_COL_H = E_LEVELS * NT, E_COL_M = E_COL_H + NT;
constexpr int E_TMEM_COLS = 512;
constexpr int E_MMAS = EMU_P * (EMU_P + 1) / 2;  // 36 products per K step

struct EBars {
    uint64_t full[NSE], empty[NSE], acc_full, acc_empty, done;
    uint32_t tmem_slot;
    int abort_flag;
};
static_assert(sizeof(EBars) <= BAR_BYTES, "barrier block");
constexpr int E_LWORDS = MT * NT * 4;         // 32 KB: the three-float sums' smallest words
static_assert(NSE * E_STAGE + E_LWORDS + BAR_BYTES <= 227 * 1024, "shared memory per CTA");
static_assert(E_COL_M + NT <= E_TMEM_COLS, "tensor memory columns");

struct EmuArgs {
    int n_tiles;
    const int64_t *kstart;     // chunk range of each tile (n_tiles + 1)
    const int2 *chunks;        // (A panel entry, B panel entry) per chunk
    const uint8_t *meta;       // per chunk: bit 0 starts a scale period, bit 1 ends one
    const int32_t *cidx;       // C block of each (M slot, N slot) pair of each tile
    const uint8_t *panel_a;    // A panels of entries [ea0, ...)
    int64_t ea0;
    const uint8_t *panel_b;    // all B panels
    const int16_t *scale_a;    // group exponent of every (A entry, row): n_ga x 128
    const int16_t *scale_b;    // group exponent of every (B entry, column): n_hb x 64
    double *C;
    int c_stride;
    double alpha, beta;
    int32_t *flag;
};

__device__ __forceinline__ uint64_t emu_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;     // leading (K) byte offset: adjacent core matrices
    d |= (uint64_t)(E_SBO >> 4) << 32;   // stride (M/N) byte offset between 8-row groups
    d |= (uint64_t)1 << 46;
    return d;
}

// x 2^e for an FP32 x, exact while the result stays a normal FP32 number
__device__ __forceinline__ float mul_pow2(float x, int e)
{
    while (e > 127) {
        x *= 1.7014118e38f;  // 2^127
        e -= 127;
    }
    while (e < -126) {
        x *= 1.1754944e-38f;  // 2^-126
        e += 126;
    }
    return x * __uint_as_float((uint32_t)(e + 127) << 23);
}

// (h, m, l) += x: two error-free sums pass the rounding errors down one word each
__device__ __forceinline__ void tf_add(float &h, float &m, float &l, float x)
{
    float s = h + x, bp = s - h;
    const float e1 = (h - (s - bp)) + (x - bp);
    h = s;
    s = m + e1;
    bp = s - m;
    const float e2 = (m - (s - bp)) + (e1 - bp);
    m = s;
    l += e2;
}

__device__ __forceinline__ void tm_ld16(uint32_t addr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
}

__device__ __forceinline__ void tm_st16(uint32_t addr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
        "%12,%13,%14,%15,%16};" ::"r"(addr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

constexpr uint8_t PERIOD_FIRST = 1, PERIOD_LAST = 2;

__device__ __forceinline__ void tm_ld8(uint32_t addr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
}

__device__ __forceinline__ void tm_st8(uint32_t addr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7])
                 : "memory");
}

template <int NB>
__global__ void __launch_bounds__(ST, 1) k_bsmm_emu(const EmuArgs p)
{
    constexpr int GI = MT / NB, GJ = NT / NB;
    extern __shared__ __align__(1024) uint8_t smem[];
    float *lws = reinterpret_cast<float *>(smem + NSE * E_STAGE);  // [column][row]
    EBars *bars = reinterpret_cast<EBars *>(smem + NSE * E_STAGE + E_LWORDS);
    volatile int *abort_flag = &bars->abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t sm0 = smem_u32(smem);

    if (t == 0) {
        for (int s = 0; s < NSE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->full[s])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->empty[s])),
                         "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->acc_full)),
                     "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->acc_empty)),
                     "r"(N_DRAIN));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->done)), "r"(1));
        bars->abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&bars->tmem_slot)),
                     "r"(E_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = bars->tmem_slot;

    if (warp == W_PROD) {
        // ------------------------------------------------------------ producer
        uint32_t sg = 0;  // running stage (K step) counter
        int last[NSE];
#pragma unroll
        for (int s = 0; s < NSE; ++s) last[s] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t c0 = p.kstart[tile];
            const int nch = (int)(p.kstart[tile + 1] - c0);
            int2 ent = make_int2(0, 0);
            for (int c = 0; c < nch && ok; ++c) {
                if ((c & 31) == 0) ent = c + lane < nch ? p.chunks[c0 + c + lane] : make_int2(0, 0);
                const int ea = __shfl_sync(0xffffffffu, ent.x, c & 31);
                const int eb = __shfl_sync(0xffffffffu, ent.y, c & 31);
                for (int ks = 0; ks < KSTEPS; ++ks, ++sg) {
                    int go = 1;
                    if (lane == 0) {
                        const int s = (int)(sg % NSE);
                        if (sg >= (uint32_t)NSE &&
                            !bar_wait(smem_u32(&bars->empty[s]), ((sg / NSE) + 1) & 1u, abort_flag)) {
                            go = 0;
                        } else {
                            const uint32_t fb = smem_u32(&bars->full[s]);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                         "r"((uint32_t)E_STAGE)
                                         : "memory");
                            bulk_copy(sm0 + s * E_STAGE,
                                      p.panel_a + (int64_t)(ea - p.ea0) * E_APANEL + ks * E_AKSTEP,
                                      E_AKSTEP, fb);
                            bulk_copy(sm0 + s * E_STAGE + E_AKSTEP,
                                      p.panel_b + (int64_t)eb * E_BPANEL + ks * E_BKSTEP, E_BKSTEP, fb);
                            last[s] = (int)sg;
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, go, 0)) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        if (lane == 0)  // every copy lands before the CTA's shared memory is released
            for (int s = 0; s < NSE; ++s)
                if (last[s] >= 0 && !bar_wait_plain(smem_u32(&bars->full[s]), (last[s] / NSE) & 1))
                    *abort_flag = 1;
        __syncwarp();
    } else if (warp == W_MMA) {
        // ------------------------------------------------------------ MMA issue
        // the warp walks the chunks (its lanes load the period flags 32 chunks at a time);
        // lane 0 waits and issues
        uint32_t sg = 0, pg = 0;
        bool ok = true, issued = false;
        const uint64_t da0 = emu_desc(sm0), db0 = emu_desc(sm0 + E_AKSTEP);
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t c0 = p.kstart[tile];
            const int nch = (int)(p.kstart[tile + 1] - c0);
            uint32_t mine = 0;
            for (int c = 0; c < nch && ok; ++c) {
                if ((c & 31) == 0) mine = c + lane < nch ? p.meta[c0 + c + lane] : 0u;
                const uint32_t meta = __shfl_sync(0xffffffffu, mine, c & 31);
                const bool first = (meta & PERIOD_FIRST) != 0;
                int go = 1;
                if (lane == 0) {
                    if (first && pg > 0 &&
                        !bar_wait(smem_u32(&bars->acc_empty), (pg - 1) & 1u, abort_flag))
                        go = 0;
                    for (int ks = 0; ks < KSTEPS && go; ++ks, ++sg) {
                        const int s = (int)(sg % NSE);
                        if (!bar_wait(smem_u32(&bars->full[s]), (sg / NSE) & 1u, abort_flag)) {
                            go = 0;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t sa = da0 + (uint64_t)((s * E_STAGE) >> 4);
                        const uint64_t sb = db0 + (uint64_t)((s * E_STAGE) >> 4);
                        // level by level (p + q ascending): back to back, the tensor cores
                        // take these 36 products faster in this order than plane by plane
#pragma unroll
                        for (int lv = 0; lv < EMU_P; ++lv)
#pragma unroll
                            for (int pa = 0; pa <= lv; ++pa) {
                                const int qb = lv - pa;
                                const int lev = lv < E_LEVELS - 1 ? lv : E_LEVELS - 1;
                                const uint64_t ad = sa + (uint64_t)((pa * E_APLANE) >> 4);
                                const uint64_t bd = sb + (uint64_t)((qb * E_BPLANE) >> 4);
                                // the first product into each accumulator of a period
                                // overwrites it: (0, l) for l < 6 in this order
                                const uint32_t acc =
                                    (first && ks == 0 && pa == 0 && lv < E_LEVELS) ? 0u : 1u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                        tmem + (uint32_t)(lev * NT)),
                                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                            }
                        bar_commit(smem_u32(&bars->empty[s]));
                        issued = true;
                    }
                    if (go && (meta & PERIOD_LAST)) bar_commit(smem_u32(&bars->acc_full));
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    ok = false;
                    break;
                }
                if (meta & PERIOD_LAST) ++pg;
            }
        }
        if (lane == 0 && issued) {  // retire every MMA before the tensor memory is released
            bar_commit(smem_u32(&bars->done));
            if (!bar_wait_plain(smem_u32(&bars->done), 0u)) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ drain and epilogue
        // the warp walks the chunks like the MMA warp (flags and panel entries 32 at a time);
        // at every chunk that ends a period it drains the accumulators with the scales of
        // that chunk's entries (all entries of one atom group in one scale group share them)
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int arow = quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
        uint32_t pg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t c0 = p.kstart[tile];
            const int nch = (int)(p.kstart[tile + 1] - c0);
            // the smallest words of this thread's row and 32 columns start at zero per tile
#pragma unroll
            for (int x = 0; x < 32; ++x) lws[(half * 32 + x) * MT + arow] = 0.f;
            bool first_period = true;
            uint32_t mine = 0;
            int2 ment = make_int2(0, 0);
            for (int c = 0; c < nch && ok; ++c) {
                if ((c & 31) == 0) {
                    mine = c + lane < nch ? p.meta[c0 + c + lane] : 0u;
                    ment = c + lane < nch ? p.chunks[c0 + c + lane] : make_int2(0, 0);
                }
                const uint32_t meta = __shfl_sync(0xffffffffu, mine, c & 31);
                const int ea_ent = __shfl_sync(0xffffffffu, ment.x, c & 31);
                const int eb_ent = __shfl_sync(0xffffffffu, ment.y, c & 31);
                if (!(meta & PERIOD_LAST)) continue;
                // scales first, so their loads overlap the wait for the accumulators
                const int ea = p.scale_a[(int64_t)ea_ent * MT + arow];
                const int4 *sb4 =
                    reinterpret_cast<const int4 *>(p.scale_b + (int64_t)eb_ent * NT + half * 32);
                const int4 s0 = __ldg(sb4), s1 = __ldg(sb4 + 1), s2 = __ldg(sb4 + 2),
                           s3 = __ldg(sb4 + 3);
                if (!bar_wait(smem_u32(&bars->acc_full), pg & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const bool last_period = (c == nch - 1);
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {  // eight columns at a time
                    const int col0 = half * 32 + q * 8;
                    const int4 sq = q == 0 ? s0 : q == 1 ? s1 : q == 2 ? s2 : s3;
                    const uint32_t su[4] = {(uint32_t)sq.x, (uint32_t)sq.y, (uint32_t)sq.z,
                                            (uint32_t)sq.w};
                    uint32_t h[8], m[8], v[E_LEVELS][8];
                    if (!first_period) {
                        tm_ld8(lane_addr + E_COL_H + q * 8, h);
                        tm_ld8(lane_addr + E_COL_M + q * 8, m);
                    }
#pragma unroll
                    for (int lev = 0; lev < E_LEVELS; ++lev)
                        tm_ld8(lane_addr + (uint32_t)(lev * NT) + q * 8, v[lev]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (first_period) {
#pragma unroll
                        for (int x = 0; x < 8; ++x) h[x] = m[x] = 0u;
                    }
#pragma unroll
                    for (int x = 0; x < 8; ++x) {
                        const int ebx = (int)(int16_t)(su[x >> 1] >> (16 * (x & 1)));
                        // a poisoned group's NaN digits made the accumulator NaN: pass it
                        // on; groups without a nonzero value contribute nothing
                        const bool poison = ea == EMU_POISON || ebx == EMU_POISON;
                        if (!poison && (ea == EMU_NONE || ebx == EMU_NONE)) continue;
                        const int e = poison ? 0 : ea + ebx - 14;
                        // the three words in registers for the six additions (the smallest
                        // one lives in shared memory between periods)
                        float hh = __uint_as_float(h[x]), mm = __uint_as_float(m[x]);
                        float ll = lws[(col0 + x) * MT + arow];
                        if (e >= -126 && e <= 127) {  // one exact scale factor for all levels
                            const float sc = __uint_as_float((uint32_t)(e + 127) << 23);
#pragma unroll
                            for (int lev = 0; lev < E_LEVELS; ++lev)
                                tf_add(hh, mm, ll, __uint_as_float(v[lev][x]) * sc);
                        } else {
#pragma unroll
                            for (int lev = 0; lev < E_LEVELS; ++lev)
                                tf_add(hh, mm, ll, mul_pow2(__uint_as_float(v[lev][x]), e));
                        }
                        lws[(col0 + x) * MT + arow] = ll;
                        h[x] = __float_as_uint(hh);
                        m[x] = __float_as_uint(mm);
                    }
                    if (!last_period) {
                        tm_st8(lane_addr + E_COL_H + q * 8, h);
                        tm_st8(lane_addr + E_COL_M + q * 8, m);
                    } else if (arow < GI * NB) {
                        // the tile's last period: C = beta C + alpha (h + m + l) in FP64
                        const int si = arow / NB, a = arow % NB;
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            const int col = col0 + x, jl = col / NB, bo = col % NB;
                            if (jl >= GJ) continue;
                            const int32_t blk = __ldg(&p.cidx[((int64_t)tile * GI + si) * GJ + jl]);
                            if (blk < 0) continue;
                            double *dst = p.C + (int64_t)blk * p.c_stride + a * NB + bo;
                            const double vv = ((double)__uint_as_float(h[x]) +
                                               (double)__uint_as_float(m[x])) +
                                              (double)lws[(col0 + x) * MT + arow];
                            *dst = p.beta == 0.0 ? p.alpha * vv : p.beta * *dst + p.alpha * vv;
                        }
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                bar_arrive(smem_u32(&bars->acc_empty));
                ++pg;
                first_period = false;
            }
            if (!ok) break;
            if (nch == 0 && arow < GI * NB) {
                // a tile without chunks: its C blocks get beta C
                const int si = arow / NB, a = arow % NB;
                for (int x = 0; x < 32; ++x) {
                    const int col = half * 32 + x, jl = col / NB, bo = col % NB;
                    if (jl >= GJ) continue;
                    const int32_t blk = __ldg(&p.cidx[((int64_t)tile * GI + si) * GJ + jl]);
                    if (blk < 0) continue;
                    double *dst = p.C + (int64_t)blk * p.c_stride + a * NB + bo;
                    *dst = p.beta == 0.0 ? 0.0 : p.beta * *dst;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (t == 0 && *abort_flag) atomicOr(p.flag, 16);
    if (warp == W_MMA) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(E_TMEM_COLS));
    }
}
