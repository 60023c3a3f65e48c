// Device-built (i, k, j) task lists of the masked product mask_{P_C}(A.B), and block maps
// between patterns.
//
// For C block (i, j) the tasks are every k with (i, k) in P_A and (k, j) in P_B, in
// ascending k.  Every pattern is symmetric, so (k, j) in P_B <=> k in row j of P_B: the
// k set is the intersection of two sorted rows.  A task is stored as the pair
// (index of block (i, k) in P_A, index of block (k, j) in P_B) -- the latter through P_B's
// transpose map -- so the product kernels never search.
#include "cq_internal.cuh"

namespace {

__device__ __forceinline__ int64_t lower_bound(const int32_t *col, int64_t lo, int64_t hi,
                                               int key)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// One warp per C block.  Writes the number of tasks and sum_k nb[k] (for the flop count).
__global__ void k_task_count(int64_t n_c, const int32_t *c_row, const int32_t *c_col,
                             const int64_t *a_rp, const int32_t *a_col, const int64_t *b_rp,
                             const int32_t *b_col, const int32_t *nb, int64_t *cnt,
                             int64_t *kw)
{
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_c) return;
    const int i = c_row[c], j = c_col[c];
    int64_t a0 = a_rp[i], a1 = a_rp[i + 1], b0 = b_rp[j], b1 = b_rp[j + 1];
    const bool walk_a = (a1 - a0) <= (b1 - b0);
    const int32_t *wc = walk_a ? a_col : b_col;
    const int32_t *sc = walk_a ? b_col : a_col;
    const int64_t w0 = walk_a ? a0 : b0, w1 = walk_a ? a1 : b1;
    const int64_t s0 = walk_a ? b0 : a0, s1 = walk_a ? b1 : a1;
    int64_t n = 0, w = 0;
    for (int64_t e = w0 + lane; e < w1; e += 32) {
        const int k = wc[e];
        const int64_t pos = lower_bound(sc, s0, s1, k);
        if (pos < s1 && sc[pos] == k) {
            ++n;
            w += nb[k];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if (lane == 0) {
        cnt[c] = n;
        kw[c] = 2 * (int64_t)nb[i] * nb[j] * w;
    }
}

__global__ void k_task_fill(int64_t n_c, const int32_t *c_row, const int32_t *c_col,
                            const int64_t *a_rp, const int32_t *a_col, const int64_t *b_rp,
                            const int32_t *b_col, const int64_t *b_tr, const int64_t *seg,
                            int2 *tasks)
{
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_c) return;
    const int i = c_row[c], j = c_col[c];
    const int64_t a0 = a_rp[i], a1 = a_rp[i + 1], b0 = b_rp[j], b1 = b_rp[j + 1];
    const bool walk_a = (a1 - a0) <= (b1 - b0);
    const int32_t *wc = walk_a ? a_col : b_col;
    const int32_t *sc = walk_a ? b_col : a_col;
    const int64_t w0 = walk_a ? a0 : b0, w1 = walk_a ? a1 : b1;
    const int64_t s0 = walk_a ? b0 : a0, s1 = walk_a ? b1 : a1;
    int64_t out = seg[c];
    for (int64_t base = w0; base < w1; base += 32) {
        const int64_t e = base + lane;
        bool hit = false;
        int64_t a_idx = 0, b_pos = 0;
        if (e < w1) {
            const int k = wc[e];
            const int64_t pos = lower_bound(sc, s0, s1, k);
            if (pos < s1 && sc[pos] == k) {
                hit = true;
                a_idx = walk_a ? e : pos;
                b_pos = walk_a ? pos : e;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int rank = __popc(m & ((1u << lane) - 1u));
            tasks[out + rank] = make_int2((int)a_idx, (int)b_tr[b_pos]);
        }
        out += __popc(m);
    }
}

__global__ void k_row_items(int64_t n_c, const int32_t *c_row, const int32_t *nb, int64_t *it)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_c) it[c] = nb[c_row[c]];
}

__global__ void k_map(int64_t n_dst, const int32_t *d_row, const int32_t *d_col,
                      const int64_t *s_rp, const int32_t *s_col, int transpose, int64_t *map)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_dst) return;
    const int i = transpose ? d_col[b] : d_row[b];
    const int j = transpose ? d_row[b] : d_col[b];
    const int64_t lo = s_rp[i], hi = s_rp[i + 1];
    const int64_t pos = lower_bound(s_col, lo, hi, j);
    map[b] = (pos < hi && s_col[pos] == j) ? pos : -1;
}

}  // namespace

cq_status cq_get_tasks(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                       const cq_pattern *pC, TaskList **out)
{
    auto key = std::make_tuple(pA->id, pB->id, pC->id);
    auto it = ctx->tasks.find(key);
    if (it != ctx->tasks.end()) {
        *out = it->second.get();
        return CQ_OK;
    }
    std::unique_ptr<TaskList> tl(new TaskList());
    const int64_t n_c = pC->n_blocks;
    tl->n_c = n_c;
    cudaStream_t s = ctx->stream;
    cq_status st;
    void *v_cnt, *v_kw, *v_kws;
    if ((st = cq_alloc(ctx, tl->seg, sizeof(int64_t) * (n_c + 1))) != CQ_OK) return st;
    if ((st = cq_scratch(ctx, "tk_cnt", sizeof(int64_t) * (n_c + 1), &v_cnt)) != CQ_OK ||
        (st = cq_scratch(ctx, "tk_kw", sizeof(int64_t) * (n_c + 1), &v_kw)) != CQ_OK ||
        (st = cq_scratch(ctx, "tk_kws", sizeof(int64_t) * (n_c + 1), &v_kws)) != CQ_OK)
        return st;
    const unsigned grid = (unsigned)((n_c + 7) / 8);
    const int32_t *nb = pA->geo->nb.as<int32_t>();
    if (n_c > 0) {
        k_task_count<<<grid, 256, 0, s>>>(n_c, pC->row.as<int32_t>(), pC->col.as<int32_t>(),
                                          pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
                                          pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), nb,
                                          (int64_t *)v_cnt, (int64_t *)v_kw);
        cq_count_launch();
    }
    if ((st = cq_scan_i64(ctx, (int64_t *)v_cnt, tl->seg.as<int64_t>(), n_c)) != CQ_OK) return st;
    if ((st = cq_scan_i64(ctx, (int64_t *)v_kw, (int64_t *)v_kws, n_c)) != CQ_OK) return st;
    int64_t tot[2] = {0, 0};
    cudaMemcpyAsync(&tot[0], tl->seg.as<int64_t>() + n_c, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&tot[1], (int64_t *)v_kws + n_c, 8, cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "task count")) != CQ_OK) return st;
    tl->n_tasks = tot[0];
    tl->flops = (double)tot[1];
    // the (A block, B block) pairs themselves are filled on the first FP64 product
    // (cq_fill_tasks): tensor-core products need only the counts, and the pairs of the long
    // products are the largest scratch of all (8 bytes per triplet)
    const int nbu = pC->geo->uniform_nb;
    if (nbu == 9 || nbu == 4) {
        tl->n_items = n_c * nbu;
    } else if (n_c > 0) {
        // prefix of block rows for the general kernel (any basis other than 4 or 9)
        void *v_items;
        if ((st = cq_scratch(ctx, "tk_items", sizeof(int64_t) * n_c, &v_items)) != CQ_OK) return st;
        if ((st = cq_alloc(ctx, tl->c_rowitem, sizeof(int64_t) * (n_c + 1))) != CQ_OK) return st;
        k_row_items<<<(unsigned)((n_c + 255) / 256), 256, 0, s>>>(n_c, pC->row.as<int32_t>(), nb,
                                                                (int64_t *)v_items);
        cq_count_launch();
        if ((st = cq_scan_i64(ctx, (int64_t *)v_items, tl->c_rowitem.as<int64_t>(), n_c)) != CQ_OK)
            return st;
        cudaMemcpyAsync(&tl->n_items, tl->c_rowitem.as<int64_t>() + n_c, sizeof(int64_t),
                        cudaMemcpyDeviceToHost, s);
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "task rows")) != CQ_OK) return st;
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "task build")) != CQ_OK) return st;
    *out = tl.get();
    ctx->tasks[key] = std::move(tl);
    return CQ_OK;
}

cq_status cq_fill_tasks(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                        const cq_pattern *pC, TaskList *tl)
{
    if (tl->filled) return CQ_OK;
    cq_status st;
    if ((st = cq_alloc(ctx, tl->tasks, sizeof(int2) * (tl->n_tasks + 1))) != CQ_OK) return st;
    const int64_t n_c = tl->n_c;
    if (n_c > 0) {
        k_task_fill<<<(unsigned)((n_c + 7) / 8), 256, 0, ctx->stream>>>(
            n_c, pC->row.as<int32_t>(), pC->col.as<int32_t>(), pA->row_ptr.as<int64_t>(),
            pA->col.as<int32_t>(), pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(),
            pB->transpose.as<int64_t>(), tl->seg.as<int64_t>(), tl->tasks.as<int2>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "task fill")) != CQ_OK) return st;
    tl->filled = true;
    return CQ_OK;
}

cq_status cq_get_map(cq_ctx *ctx, const cq_pattern *pSrc, const cq_pattern *pDst,
                     int transpose, const int64_t **out)
{
    if (pSrc == pDst && transpose) {
        *out = pSrc->transpose.as<int64_t>();
        return CQ_OK;
    }
    auto key = std::make_tuple(pSrc->id, pDst->id, transpose);
    auto it = ctx->maps.find(key);
    if (it != ctx->maps.end()) {
        *out = it->second->as<int64_t>();
        return CQ_OK;
    }
    std::unique_ptr<DevBuf> m(new DevBuf());
    cq_status st = cq_alloc(ctx, *m, sizeof(int64_t) * (pDst->n_blocks + 1));
    if (st != CQ_OK) return st;
    if (pDst->n_blocks > 0) {
        k_map<<<(unsigned)((pDst->n_blocks + 255) / 256), 256, 0, ctx->stream>>>(
            pDst->n_blocks, pDst->row.as<int32_t>(), pDst->col.as<int32_t>(),
            pSrc->row_ptr.as<int64_t>(), pSrc->col.as<int32_t>(), transpose, m->as<int64_t>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "block map")) != CQ_OK) return st;
    *out = m->as<int64_t>();
    ctx->maps[key] = std::move(m);
    return CQ_OK;
}
