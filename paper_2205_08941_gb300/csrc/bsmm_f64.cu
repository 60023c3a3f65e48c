// FP64 block-sparse product C <- beta C + alpha mask_{P_C}(A.B) on FP64 FMAs.
//
// Work decomposition: an "item" is one scalar row r of one C block c; Q adjacent lanes of
// a warp share an item and split its task segment (lane q takes tasks q, q+Q, ...), each
// keeping the item's NB partial sums in registers; the Q partials are then combined by a
// fixed xor-shuffle tree, so every C row has exactly one writer (no atomics) and the
// summation order is fixed (deterministic).  Q is picked from the mean segment length so
// that long segments (k-sums of ~800 blocks) keep all 32 lanes busy and short ones (~13)
// do not idle lanes.  The B block of a task is read by the NB lanes that own the rows of
// the same C block, so it is served from L1 after the first touch.
#include "cq_internal.cuh"

namespace {

template <int NB, int Q>
__global__ void __launch_bounds__(256)
k_bsmm_f64_uniform(int64_t n_items, const int64_t *__restrict__ seg,
                   const int2 *__restrict__ tasks, const double *__restrict__ A,
                   const double *__restrict__ B, double *__restrict__ C, int stride,
                   double alpha, double beta)
{
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t item = gt / Q;
    const int q = (int)(gt % Q);
    const bool active = item < n_items;
    const int64_t c = active ? item / NB : 0;
    const int r = (int)(item % NB);
    double acc[NB];
#pragma unroll
    for (int x = 0; x < NB; ++x) acc[x] = 0.0;
    if (active) {
        const int64_t t1 = seg[c + 1];
        for (int64_t t = seg[c] + q; t < t1; t += Q) {
            const int2 tk = __ldg(&tasks[t]);
            const double *a = A + (int64_t)tk.x * stride + r * NB;
            const double *b = B + (int64_t)tk.y * stride;
            double av[NB];
#pragma unroll
            for (int m = 0; m < NB; ++m) av[m] = __ldg(a + m);
#pragma unroll
            for (int m = 0; m < NB; ++m)
#pragma unroll
                for (int x = 0; x < NB; ++x) acc[x] = fma(av[m], __ldg(b + m * NB + x), acc[x]);
        }
    }
#pragma unroll
    for (int o = Q >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int x = 0; x < NB; ++x) acc[x] += __shfl_xor_sync(0xffffffffu, acc[x], o);
    if (active && q == 0) {
        double *cp = C + c * stride + r * NB;
        if (beta == 0.0) {
#pragma unroll
            for (int x = 0; x < NB; ++x) cp[x] = alpha * acc[x];
        } else {
#pragma unroll
            for (int x = 0; x < NB; ++x) cp[x] = beta * cp[x] + alpha * acc[x];
        }
    }
}

// One C row of the mixed-basis product with NJ columns: the Q lanes of the row's group take
// tasks q, q + Q, ..., keep NJ partial sums and combine them with a fixed xor tree over the
// group (gmask: the group's lanes, so that groups of different widths may branch apart).
// NJ == CQ_MAX_NB is the catch-all for widths without their own instance (nj_rt columns).
template <int NJ, int Q>
__device__ __forceinline__ void generic_row(unsigned gmask, int q, int64_t c, int r, int ni,
                                            int nj_rt, const int64_t *__restrict__ seg,
                                            const int2 *__restrict__ tasks,
                                            const int32_t *__restrict__ nb,
                                            const int32_t *__restrict__ a_col,
                                            const int64_t *__restrict__ a_off,
                                            const int64_t *__restrict__ b_off,
                                            const int64_t *__restrict__ c_off,
                                            const double *__restrict__ A,
                                            const double *__restrict__ B, double *__restrict__ C,
                                            double alpha, double beta)
{
    constexpr bool ANY = NJ == CQ_MAX_NB;
    const int nj = ANY ? nj_rt : NJ;
    double acc[NJ];
#pragma unroll
    for (int x = 0; x < NJ; ++x) acc[x] = 0.0;
    const int64_t t1 = seg[c + 1];
    for (int64_t t = seg[c] + q; t < t1; t += Q) {
        const int2 tk = __ldg(&tasks[t]);
        const int nk = nb[a_col[tk.x]];
        const double *a = A + a_off[tk.x] + (int64_t)r * nk;
        const double *b = B + b_off[tk.y];
        for (int m = 0; m < nk; ++m) {
            const double av = __ldg(a + m);
#pragma unroll
            for (int x = 0; x < NJ; ++x)
                if (!ANY || x < nj) acc[x] = fma(av, __ldg(b + m * nj + x), acc[x]);
        }
    }
#pragma unroll
    for (int o = Q >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int x = 0; x < NJ; ++x) acc[x] += __shfl_xor_sync(gmask, acc[x], o);
    if (q == 0 && r < ni) {
        double *cp = C + c_off[c] + (int64_t)r * nj;
#pragma unroll
        for (int x = 0; x < NJ; ++x)
            if (!ANY || x < nj)
                cp[x] = (beta == 0.0) ? alpha * acc[x] : beta * cp[x] + alpha * acc[x];
    }
}

// Mixed orbital counts (1..16 per atom): item -> C block by binary search over the prefix
// of block row counts; block offsets from the patterns' val_off.  The row's column count
// selects an instance with exactly that many accumulators (4, 5, 9, 13: the bases of the
// mixed-species cells), so no FMA slot or shuffle is spent on absent columns.
template <int Q>
__global__ void __launch_bounds__(256)
k_bsmm_f64_generic(int64_t n_items, int64_t n_c, const int64_t *__restrict__ rowitem,
                   const int64_t *__restrict__ seg, const int2 *__restrict__ tasks,
                   const int32_t *__restrict__ nb, const int32_t *__restrict__ c_row,
                   const int32_t *__restrict__ c_col, const int32_t *__restrict__ a_col,
                   const int64_t *__restrict__ a_off, const int64_t *__restrict__ b_off,
                   const int64_t *__restrict__ c_off, const double *__restrict__ A,
                   const double *__restrict__ B, double *__restrict__ C, double alpha,
                   double beta)
{
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t item = gt / Q;
    const int q = (int)(gt % Q);
    if (item >= n_items) return;  // whole Q groups leave together (blockDim is a multiple of Q)
    int64_t lo = 0, hi = n_c;     // largest c with rowitem[c] <= item
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (rowitem[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    const int64_t c = lo;
    const int r = (int)(item - rowitem[c]);
    const int ni = nb[c_row[c]], nj = nb[c_col[c]];
    const unsigned gmask =
        Q == 32 ? 0xffffffffu : (((1u << Q) - 1u) << ((threadIdx.x & 31) & ~(Q - 1)));
#define CQ_ROW(NJ)                                                                           \
    generic_row<NJ, Q>(gmask, q, c, r, ni, nj, seg, tasks, nb, a_col, a_off, b_off, c_off, A, \
                       B, C, alpha, beta)
    switch (nj) {
    case 4: CQ_ROW(4); break;
    case 5: CQ_ROW(5); break;
    case 9: CQ_ROW(9); break;
    case 13: CQ_ROW(13); break;
    default: CQ_ROW(CQ_MAX_NB); break;
    }
#undef CQ_ROW
}

int pick_q(const TaskList *tl)
{
    const double avg = tl->n_c ? (double)tl->n_tasks / (double)tl->n_c : 0.0;
    int q = 1;
    while (q < 32 && q * 8 <= avg) q <<= 1;
    return q;
}

template <int NB>
void launch_uniform(int q, unsigned grid, cudaStream_t s, int64_t n_items, const TaskList *tl,
                    const double *A, const double *B, double *C, int stride, double alpha,
                    double beta)
{
    const int64_t *seg = tl->seg.as<int64_t>();
    const int2 *tk = tl->tasks.as<int2>();
#define CQ_LAUNCH(QQ)                                                                      \
    k_bsmm_f64_uniform<NB, QQ><<<grid, 256, 0, s>>>(n_items, seg, tk, A, B, C, stride, alpha, \
                                                    beta)
    switch (q) {
    case 1: CQ_LAUNCH(1); break;
    case 2: CQ_LAUNCH(2); break;
    case 4: CQ_LAUNCH(4); break;
    case 8: CQ_LAUNCH(8); break;
    case 16: CQ_LAUNCH(16); break;
    default: CQ_LAUNCH(32); break;
    }
#undef CQ_LAUNCH
}

}  // namespace

// One launch of the FP64 product with lane split q.
static void launch_f64(cq_ctx *ctx, int q, const TaskList *tl, double alpha,
                       const cq_pattern *pA, const double *A, const cq_pattern *pB,
                       const double *B, double beta, const cq_pattern *pC, double *C)
{
    const int nbu = pC->geo->uniform_nb;
    cudaStream_t s = ctx->stream;
    const int64_t n_items = tl->n_items;
    const unsigned grid = (unsigned)((n_items * q + 255) / 256);
    if (nbu == 9 || nbu == 4) {
        if (nbu == 9)
            launch_uniform<9>(q, grid, s, n_items, tl, A, B, C, pC->uniform, alpha, beta);
        else
            launch_uniform<4>(q, grid, s, n_items, tl, A, B, C, pC->uniform, alpha, beta);
        return;
    }
    const int64_t *rowitem = tl->c_rowitem.as<int64_t>();
    const int32_t *nb = pC->geo->nb.as<int32_t>();
#define CQ_GEN(QQ)                                                                            \
    k_bsmm_f64_generic<QQ><<<grid, 256, 0, s>>>(                                              \
        n_items, tl->n_c, rowitem, tl->seg.as<int64_t>(), tl->tasks.as<int2>(), nb,           \
        pC->row.as<int32_t>(), pC->col.as<int32_t>(), pA->col.as<int32_t>(),                  \
        pA->val_off.as<int64_t>(), pB->val_off.as<int64_t>(), pC->val_off.as<int64_t>(), A, B, \
        C, alpha, beta)
    switch (q) {
    case 1: CQ_GEN(1); break;
    case 2: CQ_GEN(2); break;
    case 4: CQ_GEN(4); break;
    case 8: CQ_GEN(8); break;
    case 16: CQ_GEN(16); break;
    default: CQ_GEN(32); break;
    }
#undef CQ_GEN
}

// Autotuner: on the first product of a task list (with autotuning on and no capture open),
// time every lane split on the real operands into scratch (beta = 0, so the caller's C is
// untouched) and keep the fastest for this task list.
static cq_status tune_q(cq_ctx *ctx, const TaskList *tl, const cq_pattern *pA, const double *A,
                        const cq_pattern *pB, const double *B, const cq_pattern *pC)
{
    void *tmp;
    cq_status st = cq_scratch(ctx, "tune_C", sizeof(double) * pC->n_values, &tmp);
    if (st != CQ_OK) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_q = pick_q(tl);
    for (int q = 1; q <= 32; q <<= 1) {
        launch_f64(ctx, q, tl, 1.0, pA, A, pB, B, 0.0, pC, (double *)tmp);  // warm
        cudaEventRecord(e0, ctx->stream);
        launch_f64(ctx, q, tl, 1.0, pA, A, pB, B, 0.0, pC, (double *)tmp);
        cudaEventRecord(e1, ctx->stream);
        cq_count_launch(2);
        st = cq_check_cuda(ctx, cudaEventSynchronize(e1), "autotune");
        if (st != CQ_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_q = q;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tl->q = best_q;
    return st;
}

int cq_lane_split(const TaskList *tl) { return tl->q ? tl->q : pick_q(tl); }

cq_status cq_bsmm_f64(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                      const double *A, const cq_pattern *pB, const double *B, double beta,
                      const cq_pattern *pC, double *C)
{
    if (tl->n_c == 0) return CQ_OK;
    if (!tl->filled) {
        if (ctx->capturing)
            return cq_fail(ctx, CQ_ERR_INVALID,
                           "bsmm: first FP64 product of a triple inside a graph capture");
        cq_status st = cq_fill_tasks(ctx, pA, pB, pC, const_cast<TaskList *>(tl));
        if (st != CQ_OK) return st;
    }
    if (ctx->autotune && tl->q == 0 && !ctx->capturing) {
        cq_status st = tune_q(ctx, tl, pA, A, pB, B, pC);
        if (st != CQ_OK) return st;
    }
    cq_timing_begin(ctx, tl->flops);
    launch_f64(ctx, cq_lane_split(tl), tl, alpha, pA, A, pB, B, beta, pC, C);
    cq_timing_end(ctx);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "bsmm_f64");
}
