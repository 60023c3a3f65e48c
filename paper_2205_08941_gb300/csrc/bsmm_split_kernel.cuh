// The tile kernel of the split-BF16 product (included by bsmm_split.cu).
//
// Warp roles (10 warps, one CTA per SM):
//   warp 0      producer: a chunk is up to three consecutive K steps of a tile; lane 0
//               copies each K step's pieces (main step: two A and two B main pieces; tail
//               step: one A and one B tail piece; 18 KB either way) into the step's slot of
//               a free stage with TMA bulk copies that complete on the stage's "full"
//               barrier; the warp's lanes load the K-step table 32 entries at a time;
//   warp 1      lane 0 issues the MMAs of a chunk (6 split products per K step) into
//               one of NACC TMEM accumulators (one per drain period, in rotation) and
//               commits them to the stage's "empty" barrier, and at the end of a drain
//               period to the accumulator's "full" barrier;
//   warps 2-9   drain: every DRAIN chunks they read the FP32 accumulator (warp w: TMEM lane
//               quarter w % 4, columns 32 * ((w - 2) / 4) ..) into double-float (hi, lo)
//               sums in registers, release the accumulator, and write C after a tile's last
//               period.
// Stages rotate over one running chunk counter across all tiles of the CTA; accumulators
// over one running period counter; every wait computes its parity from those counters.
//
// Every wait is bounded (about two seconds) and also ends when another role has given up:
// the CTA then stops issuing work, retires its own copies and MMAs (bounded), frees its
// tensor memory and returns with bit 16 of the context flag set.
constexpr int NS = 4;                  // shared-memory stages
constexpr int N_DRAIN = 256;           // drain threads
constexpr int W_PROD = 0, W_MMA = 1;   // producer warp, MMA warp

struct Bars {
    uint64_t full[NS], empty[NS], acc_full[NACC], acc_empty[NACC], done;
    uint64_t never;  // no thread ever arrives here: the test-only wait on it must run out
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

// Bounded wait with its own limit in cycles (the test-only short wait).
__device__ __forceinline__ bool bar_wait_for(uint32_t addr, uint32_t parity,
                                             volatile int *abort_flag, long long limit)
{
    const long long t0 = clock64();
    while (!bar_try(addr, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
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

// TMA bulk copy global -> shared completing `bytes` of transaction count on mbarrier bar
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Epilogue of one drain thread: accumulator row arow = (atom of M slot si, orbital a),
// columns 32*HALF .. +31 = (atom of N slot, orbital); cid[u] is the P_C block of slot pair
// (si, J0 + u) or -1; each present block gets beta*C + alpha*(hi + lo).
template <int NB> __host__ __device__ constexpr int epi_slots() { return 32 / (NB ? NB : 32) + 2; }

template <int NB, int HALF>
__device__ __forceinline__ void write_rows(const SplitArgs &p, const int32_t (&cid)[epi_slots<NB>()],
                                           int arow, const float (&hi)[32], const float (&lo)[32])
{
    constexpr int GI = MT / NB, GJ = NT / NB;
    constexpr int J0 = (HALF * 32) / NB, J1 = (HALF * 32 + 31) / NB;
    if (arow >= GI * NB) return;
    const int a = arow % NB;
#pragma unroll
    for (int jl = J0; jl <= J1; ++jl) {
        if (jl >= GJ || jl - J0 >= epi_slots<NB>()) continue;
        const int32_t blk = cid[jl - J0];
        if (blk < 0) continue;
        double *dst = p.C + (int64_t)blk * p.c_stride + a * NB;
#pragma unroll
        for (int bo = 0; bo < NB; ++bo) {
            const int x = jl * NB + bo - HALF * 32;
            if (x < 0 || x >= 32) continue;
            const double v = (double)hi[x] + (double)lo[x];
            dst[bo] = p.beta == 0.0 ? p.alpha * v : p.beta * dst[bo] + p.alpha * v;
        }
    }
}

// NB = 0: mixed basis (groups, rows and columns through the tables of bsmm_mixed.cuh)
template <int NB>
__global__ void __launch_bounds__(ST, 1) k_bsmm_split(const SplitArgs p)
{
    constexpr int GI = NB ? MT / NB : GI_MIX, GJ = NB ? NT / NB : GJ_MIX;
    extern __shared__ __align__(1024) uint8_t smem[];
    Bars *bars = reinterpret_cast<Bars *>(smem + NS * STAGE);
    volatile int *abort_flag = &bars->abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t sm0 = smem_u32(smem);

    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->full[s])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->empty[s])),
                         "r"(1));
        }
        for (int b = 0; b < NACC; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                             smem_u32(&bars->acc_full[b])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                             smem_u32(&bars->acc_empty[b])),
                         "r"(N_DRAIN));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->done)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars->never)), "r"(1));
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

    if (warp == W_PROD) {
        // ------------------------------------------------------------ producer
        uint32_t cg = 0;  // running chunk counter
        int last[NS];     // last chunk issued into each stage (lane 0)
#pragma unroll
        for (int s = 0; s < NS; ++s) last[s] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int64_t s0 = p.kstart[tile];
            const int nks = (int)(p.kstart[tile + 1] - s0);
            const int nm = p.nmain[tile];
            const int nch = (nks + KSTEPS - 1) / KSTEPS;
            int4 ent = make_int4(0, 0, 0, 0);
            for (int c = 0; c < nch; ++c, ++cg) {
                const int s = (int)(cg % NS);
                const int nv = min(KSTEPS, nks - KSTEPS * c);  // K steps of this chunk
                int go = 1;
                if (lane == 0) {
                    if (cg >= (uint32_t)NS &&
                        !bar_wait(smem_u32(&bars->empty[s]), ((cg / NS) + 1) & 1u, abort_flag)) {
                        go = 0;
                    } else {
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         smem_u32(&bars->full[s])),
                                     "r"((uint32_t)(nv * (A_SLOT + B_SLOT)))
                                     : "memory");
                        last[s] = (int)cg;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    ok = false;
                    break;
                }
                for (int x = 0; x < nv; ++x) {
                    const int q = KSTEPS * c + x;
                    if ((q & 31) == 0)
                        ent = q + lane < nks ? p.steps[s0 + q + lane] : make_int4(0, 0, 0, 0);
                    const int ea = __shfl_sync(0xffffffffu, ent.x, q & 31);
                    const int ea2 = __shfl_sync(0xffffffffu, ent.y, q & 31);
                    const int eb = __shfl_sync(0xffffffffu, ent.z, q & 31);
                    const int eb2 = __shfl_sync(0xffffffffu, ent.w, q & 31);
                    if (lane == 0) {
                        const uint32_t fb = smem_u32(&bars->full[s]);
                        const uint32_t da = sm0 + s * STAGE + x * A_SLOT;
                        const uint32_t db = sm0 + s * STAGE + B_SLOTS + x * B_SLOT;
                        if (q < nm) {
                            bulk_copy(da, p.a_main + (int64_t)(ea - p.am0) * A_MAIN, A_MAIN, fb);
                            bulk_copy(da + A_MAIN,
                                      ea2 < 0 ? p.zero : p.a_main + (int64_t)(ea2 - p.am0) * A_MAIN,
                                      A_MAIN, fb);
                            bulk_copy(db, p.b_main + (int64_t)eb * B_MAIN, B_MAIN, fb);
                            bulk_copy(db + B_MAIN, eb2 < 0 ? p.zero : p.b_main + (int64_t)eb2 * B_MAIN,
                                      B_MAIN, fb);
                        } else {
                            bulk_copy(da, p.a_tail + (int64_t)(ea - p.at0) * A_TAIL, A_TAIL, fb);
                            bulk_copy(db, p.b_tail + (int64_t)eb * B_TAIL, B_TAIL, fb);
                        }
                    }
                }
            }
        }
        if (lane == 0)  // every copy lands before the CTA's shared memory is released
            for (int s = 0; s < NS; ++s)
                if (last[s] >= 0 && !bar_wait_plain(smem_u32(&bars->full[s]), (last[s] / NS) & 1))
                    *abort_flag = 1;
        __syncwarp();
    } else if (warp == W_MMA) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            uint32_t cg = 0, pg = 0;
            bool ok = true, issued = false;
            // test mode: the first wait is on a barrier nothing completes, with a short limit,
            // so it runs out; the CTA then takes the same abort path as a real timeout
            if (p.test_wait_cycles > 0) {
                bar_wait_for(smem_u32(&bars->never), 0u, abort_flag, p.test_wait_cycles);
                ok = false;
            }
            const int pq[6][2] = {{0, 0}, {0, 1}, {1, 0}, {0, 2}, {1, 1}, {2, 0}};
            // descriptors of slot 0 of stage 0 for both kinds of K step (main: the second
            // column is the second atom's piece, A_MAIN / B_MAIN further; tail: the piece's
            // second column); a stage, slot or plane only moves the 14-bit start address
            // field (shared addresses stay below 256 KB, so no carry leaves it)
            const uint64_t dam = piece_desc(sm0, A_MAIN), dat = piece_desc(sm0, COLB_A);
            const uint64_t dbm = piece_desc(sm0 + B_SLOTS, B_MAIN);
            const uint64_t dbt = piece_desc(sm0 + B_SLOTS, COLB_B);
            for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
                const int nks = (int)(p.kstart[tile + 1] - p.kstart[tile]);
                const int nm = p.nmain[tile];
                const int nch = (nks + KSTEPS - 1) / KSTEPS;
                for (int c = 0; c < nch; ++c, ++cg) {
                    const uint32_t b = pg % NACC;
                    if (c % DRAIN == 0 && pg >= (uint32_t)NACC &&
                        !bar_wait(smem_u32(&bars->acc_empty[b]), ((pg / NACC) + 1) & 1u,
                                  abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int s = (int)(cg % NS);
                    if (!bar_wait(smem_u32(&bars->full[s]), (cg / NS) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc_addr = tmem + b * NT;
                    const int nv = min(KSTEPS, nks - KSTEPS * c);
                    for (int ks = 0; ks < nv; ++ks) {
                        const bool main_step = KSTEPS * c + ks < nm;
                        // plane strides in 16-byte units: main pieces hold one column per
                        // plane, tail pieces two
                        const uint32_t pa = main_step ? COLB_A >> 4 : (2 * COLB_A) >> 4;
                        const uint32_t pb = main_step ? COLB_B >> 4 : (2 * COLB_B) >> 4;
                        const uint64_t sa = (main_step ? dam : dat) +
                                            (uint64_t)((s * STAGE + ks * A_SLOT) >> 4);
                        const uint64_t sb = (main_step ? dbm : dbt) +
                                            (uint64_t)((s * STAGE + ks * B_SLOT) >> 4);
#pragma unroll
                        for (int x = 0; x < 6; ++x) {
                            const uint64_t ad = sa + (uint64_t)(pq[x][0] * pa);
                            const uint64_t bd = sb + (uint64_t)(pq[x][1] * pb);
                            const uint32_t acc = (c % DRAIN == 0 && ks == 0 && x == 0) ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                    acc_addr),
                                "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                        }
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
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        const int arow = quarter * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 32);
        uint32_t pg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
            const int nks = (int)(p.kstart[tile + 1] - p.kstart[tile]);
            const int nch = (nks + KSTEPS - 1) / KSTEPS;
            const int np = (nch + DRAIN - 1) / DRAIN;
            // this row's C blocks, loaded now and used after the tile's last period
            constexpr int NJ = epi_slots<NB>();
            int32_t cid[NJ];
            if constexpr (NB > 0) {
                const int si = arow / NB, j0 = (half * 32) / NB;
#pragma unroll
                for (int u = 0; u < NJ; ++u)
                    cid[u] = (arow < GI * NB && j0 + u < GJ)
                                 ? __ldg(&p.cidx[((int64_t)tile * GI + si) * GJ + j0 + u])
                                 : -1;
            }
            float hi[32], lo[32];
#pragma unroll
            for (int x = 0; x < 32; ++x) hi[x] = lo[x] = 0.f;
            for (int d = 0; d < np; ++d, ++pg) {
                const uint32_t b = pg % NACC;
                if (!bar_wait(smem_u32(&bars->acc_full[b]), (pg / NACC) & 1u, abort_flag)) {
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
            if constexpr (NB > 0) {
                if (half == 0)
                    write_rows<NB, 0>(p, cid, arow, hi, lo);
                else
                    write_rows<NB, 1>(p, cid, arow, hi, lo);
            } else {
                write_rows_mixed(p, tile, arow, half, hi, lo);
            }
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
