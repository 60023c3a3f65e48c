// The tile kernel of the emulated-FP64 product (included by bsmm_split.cu after the split
// kernel, whose barrier, copy and timeout helpers it shares).
//
// Operands are eight BF16 digit planes per value (emu_digits.cuh): A_p, B_q with planes
// pre-scaled by 2^(-8p), so the MMA of planes p and q lands at level p + q.  Per K step the
// MMA thread issues the 36 products with p + q <= 7, level by level, into six FP32
// accumulators in tensor memory: levels 0 to 4 each alone -- over one scale period a
// level-l sum is an integer times 2^(-8 l) of magnitude at most (l + 1) * 144 * 128^2 < 2^24
// (at most 144 K values per period), hence exact -- and levels 5-7 together (rounded, but
// 2^-40 below level 0, so its rounding stays near 2^-64 of the group's scale, as does the
// digit split itself).  A scale period is one tail group of K (16 consecutive atoms in Morton
// order for 9 orbitals, 4 for 4): the main K steps pairing the tile's K atoms of the group,
// then the group's tail step.  At its end the drain warps scale every level by
// 2^(E_A(row) + E_B(column) - 14) and add it into a three-float sum (h, m, l): h and m in
// tensor memory beside the accumulators, l (the smallest word) in shared memory (column-
// major, so the lanes of a warp, which own consecutive rows, hit distinct banks).  After a
// tile's last period C = beta C + alpha (h + m + l) is written in FP64.
//
// Warp roles (10 warps, one CTA per SM):
//   warp 0      producer: lane 0 copies the pieces of every K step (main step: two A main
//               pieces of 8 planes x 128 rows x 8 K, 16 KB each, and two B main pieces of
//               8 KB; tail step: one A tail piece, 32 KB, and one B tail piece, 16 KB) into a
//               free stage with TMA bulk copies completing on the stage's "full" barrier;
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
constexpr int E_AMAIN = EMU_P * COLB_A;      // 16 KB: an A main piece (planes x one column)
constexpr int E_BMAIN = EMU_P * COLB_B;      // 8 KB
constexpr int E_ATAIL = 2 * E_AMAIN;         // 32 KB: an A tail piece (planes x two columns)
constexpr int E_BTAIL = 2 * E_BMAIN;         // 16 KB
constexpr int E_STAGE = E_ATAIL + E_BTAIL;   // one K step: A at 0, B at E_ATAIL
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
    const int64_t *kstart;     // K-step range of each tile (n_tiles + 1)
    const int4 *steps;         // piece entries of every K step
    const uint8_t *meta;       // per K step: bit 0 starts a scale period, bit 1 ends one
                               // (the period's tail step)
    const int32_t *cidx;       // C block of each (M slot, N slot) pair of each tile
    const uint8_t *a_main;     // A main pieces of entries [am0, ...)
    int64_t am0;
    const uint8_t *a_tail;     // A tail pieces of entries [at0, ...)
    int64_t at0;
    const uint8_t *b_main;     // all B main pieces
    const uint8_t *b_tail;     // all B tail pieces
    const uint8_t *zero;       // an all-zero A main piece
    const int16_t *scale_a;    // group exponent of every (A tail entry, row): n_at x 128
    const int16_t *scale_b;    // group exponent of every (B tail entry, column): n_bt x 64
    double *C;
    int c_stride;
    double alpha, beta;
    int32_t *flag;
};

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
            const int64_t s0 = p.kstart[tile];
            const int nks = (int)(p.kstart[tile + 1] - s0);
            int4 ent = make_int4(0, 0, 0, 0);
            uint32_t mine = 0;
            for (int q = 0; q < nks; ++q, ++sg) {
                if ((q & 31) == 0) {
                    ent = q + lane < nks ? p.steps[s0 + q + lane] : make_int4(0, 0, 0, 0);
                    mine = q + lane < nks ? p.meta[s0 + q + lane] : 0u;
                }
                const int ea = __shfl_sync(0xffffffffu, ent.x, q & 31);
                const int ea2 = __shfl_sync(0xffffffffu, ent.y, q & 31);
                const int eb = __shfl_sync(0xffffffffu, ent.z, q & 31);
                const int eb2 = __shfl_sync(0xffffffffu, ent.w, q & 31);
                const uint32_t meta = __shfl_sync(0xffffffffu, mine, q & 31);
                int go = 1;
                if (lane == 0) {
                    const int s = (int)(sg % NSE);
                    if (sg >= (uint32_t)NSE &&
                        !bar_wait(smem_u32(&bars->empty[s]), ((sg / NSE) + 1) & 1u, abort_flag)) {
                        go = 0;
                    } else {
                        const uint32_t fb = smem_u32(&bars->full[s]);
                        const uint32_t da = sm0 + s * E_STAGE, db = da + E_ATAIL;
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"((uint32_t)E_STAGE)
                                     : "memory");
                        if (meta & PERIOD_LAST) {  // tail step
                            bulk_copy(da, p.a_tail + (int64_t)(ea - p.at0) * E_ATAIL, E_ATAIL, fb);
                            bulk_copy(db, p.b_tail + (int64_t)eb * E_BTAIL, E_BTAIL, fb);
                        } else {
                            bulk_copy(da, p.a_main + (int64_t)(ea - p.am0) * E_AMAIN, E_AMAIN, fb);
                            bulk_copy(da + E_AMAIN,
                                      ea2 < 0 ? p.zero : p.a_main + (int64_t)(ea2 - p.am0) * E_AMAIN,
                                      E_AMAIN, fb);
                            bulk_copy(db, p.b_main + (int64_t)eb * E_BMAIN, E_BMAIN, fb);
                            bulk_copy(db + E_BMAIN, eb2 < 0 ? p.zero : p.b_main + (int64_t)eb2 * E_BMAIN,
                                      E_BMAIN, fb);
                        }
                        last[s] = (int)sg;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    ok = false;
                    break;
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
        // the warp walks the K steps (its lanes load the period flags 32 steps at a time);
        // lane 0 waits and issues
        uint32_t sg = 0, pg = 0;
        bool ok = true, issued = false;
        // descriptors of stage 0 for both kinds of K step (main: the second column is the
        // second atom's piece; tail: the piece's second column); a stage or plane only moves
        // the 14-bit start address field
        const uint64_t dam = piece_desc(sm0, E_AMAIN), dat = piece_desc(sm0, COLB_A);
        const uint64_t dbm = piece_desc(sm0 + E_ATAIL, E_BMAIN), dbt = piece_desc(sm0 + E_ATAIL, COLB_B);
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t s0 = p.kstart[tile];
            const int nks = (int)(p.kstart[tile + 1] - s0);
            uint32_t mine = 0;
            for (int q = 0; q < nks && ok; ++q, ++sg) {
                if ((q & 31) == 0) mine = q + lane < nks ? p.meta[s0 + q + lane] : 0u;
                const uint32_t meta = __shfl_sync(0xffffffffu, mine, q & 31);
                const bool first = (meta & PERIOD_FIRST) != 0, tail = (meta & PERIOD_LAST) != 0;
                int go = 1;
                if (lane == 0) {
                    const int s = (int)(sg % NSE);
                    if (first && pg > 0 &&
                        !bar_wait(smem_u32(&bars->acc_empty), (pg - 1) & 1u, abort_flag))
                        go = 0;
                    else if (!bar_wait(smem_u32(&bars->full[s]), (sg / NSE) & 1u, abort_flag))
                        go = 0;
                    if (go) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        // plane strides in 16-byte units: main pieces hold one column per
                        // plane, tail pieces two
                        const uint32_t pla = tail ? (2 * COLB_A) >> 4 : COLB_A >> 4;
                        const uint32_t plb = tail ? (2 * COLB_B) >> 4 : COLB_B >> 4;
                        const uint64_t sa = (tail ? dat : dam) + (uint64_t)((s * E_STAGE) >> 4);
                        const uint64_t sb = (tail ? dbt : dbm) + (uint64_t)((s * E_STAGE) >> 4);
                        // level by level (p + q ascending): back to back, the tensor cores
                        // take these 36 products faster in this order than plane by plane
#pragma unroll
                        for (int lv = 0; lv < EMU_P; ++lv)
#pragma unroll
                            for (int pa = 0; pa <= lv; ++pa) {
                                const int qb = lv - pa;
                                const int lev = lv < E_LEVELS - 1 ? lv : E_LEVELS - 1;
                                const uint64_t ad = sa + (uint64_t)(pa * pla);
                                const uint64_t bd = sb + (uint64_t)(qb * plb);
                                // the first product into each accumulator of a period
                                // overwrites it: (0, l) for l < 6 in this order
                                const uint32_t acc = (first && pa == 0 && lv < E_LEVELS) ? 0u : 1u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                        tmem + (uint32_t)(lev * NT)),
                                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                            }
                        bar_commit(smem_u32(&bars->empty[s]));
                        issued = true;
                        if (tail) bar_commit(smem_u32(&bars->acc_full));
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    ok = false;
                    break;
                }
                if (tail) ++pg;
            }
        }
        if (lane == 0 && issued) {  // retire every MMA before the tensor memory is released
            bar_commit(smem_u32(&bars->done));
            if (!bar_wait_plain(smem_u32(&bars->done), 0u)) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ drain and epilogue
        // the warp walks the K steps like the MMA warp (flags and entries 32 at a time); at
        // every tail step it drains the accumulators with the scales of the step's tail
        // pieces (the period's group exponents)
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int arow = quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
        uint32_t pg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t s0 = p.kstart[tile];
            const int nks = (int)(p.kstart[tile + 1] - s0);
            // the smallest words of this thread's row and 32 columns start at zero per tile
#pragma unroll
            for (int x = 0; x < 32; ++x) lws[(half * 32 + x) * MT + arow] = 0.f;
            bool first_period = true;
            uint32_t mine = 0;
            int4 ment = make_int4(0, 0, 0, 0);
            for (int q = 0; q < nks && ok; ++q) {
                if ((q & 31) == 0) {
                    mine = q + lane < nks ? p.meta[s0 + q + lane] : 0u;
                    ment = q + lane < nks ? p.steps[s0 + q + lane] : make_int4(0, 0, 0, 0);
                }
                const uint32_t meta = __shfl_sync(0xffffffffu, mine, q & 31);
                const int ea_ent = __shfl_sync(0xffffffffu, ment.x, q & 31);
                const int eb_ent = __shfl_sync(0xffffffffu, ment.z, q & 31);
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
                const bool last_period = (q == nks - 1);
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
            if (nks == 0 && arow < GI * NB) {
                // a tile without K steps: its C blocks get beta C
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
