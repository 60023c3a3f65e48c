// Range-cutoff pattern construction on the device: cell-list binning, per-row neighbour
// collection with a shared-memory bitonic sort, block offsets and the transpose map.
//
// P_R = {(i, j) : d_min(i, j)^2 < R^2} plus every (i, i) (the paper's locality: matrices are
// stored only for atom pairs within a range).  The squared distance is evaluated exactly as
// ((dx*dx + dy*dy) + dz*dz), d = (x_j - x_i) - box*rint((x_j - x_i)/box), with round-to-
// nearest intrinsics so that no FMA contraction can move a pair across the cutoff.
#include <cmath>
#include <cstring>

#include "cq_internal.cuh"

namespace {

constexpr int ROW_THREADS = 256;

__device__ __forceinline__ double min_image_d2(const double *pos, const double *box, int i,
                                               int j)
{
    double d2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d = __dsub_rn(pos[3 * j + c], pos[3 * i + c]);
        d = __dsub_rn(d, __dmul_rn(box[c], rint(__ddiv_rn(d, box[c]))));
        d2 = __dadd_rn(d2, __dmul_rn(d, d));
    }
    return d2;
}

struct CellGrid {
    int nc[3];
    double box[3];
};

__device__ __forceinline__ int cell_coord(double x, double box, int nc)
{
    double f = x / box;
    f = f - floor(f);
    int c = (int)(f * nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_of(int n, const double *pos, CellGrid g, int32_t *cell_of,
                          int64_t *cell_count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(pos[3 * i + 0], g.box[0], g.nc[0]);
    int cy = cell_coord(pos[3 * i + 1], g.box[1], g.nc[1]);
    int cz = cell_coord(pos[3 * i + 2], g.box[2], g.nc[2]);
    int c = (cx * g.nc[1] + cy) * g.nc[2] + cz;
    cell_of[i] = c;
    atomicAdd((unsigned long long *)&cell_count[c], 1ull);
}

__global__ void k_cell_fill(int n, const int32_t *cell_of, const int64_t *cell_start,
                            int64_t *cursor, int32_t *cell_atoms)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int64_t s = (int64_t)atomicAdd((unsigned long long *)&cursor[c], 1ull);
    cell_atoms[cell_start[c] + s] = i;
}

// One CTA per atom row.  COUNT: number of neighbours -> row_count.  FILL: neighbours sorted
// ascending -> col[row_ptr[i] ...].  Rows longer than CQ_ROW_CAP raise flag bit 1.
template <bool FILL>
__global__ void __launch_bounds__(ROW_THREADS)
k_rows(int n, const double *pos, CellGrid g, const int32_t *cell_of, const int64_t *cell_start,
       const int32_t *cell_atoms, double r2, int64_t *row_count, const int64_t *row_ptr,
       int32_t *col, int32_t *flag)
{
    __shared__ int32_t buf[FILL ? CQ_ROW_CAP : 1];
    __shared__ int count;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    const int c0 = cell_of[i];
    const int cz0 = c0 % g.nc[2], cy0 = (c0 / g.nc[2]) % g.nc[1], cx0 = c0 / (g.nc[2] * g.nc[1]);
    const int sx = g.nc[0] >= 3 ? 3 : 1, sy = g.nc[1] >= 3 ? 3 : 1, sz = g.nc[2] >= 3 ? 3 : 1;
    int local = 0;
    for (int ox = 0; ox < sx; ++ox)
        for (int oy = 0; oy < sy; ++oy)
            for (int oz = 0; oz < sz; ++oz) {
                int cx = sx == 3 ? (cx0 + ox - 1 + g.nc[0]) % g.nc[0] : cx0;
                int cy = sy == 3 ? (cy0 + oy - 1 + g.nc[1]) % g.nc[1] : cy0;
                int cz = sz == 3 ? (cz0 + oz - 1 + g.nc[2]) % g.nc[2] : cz0;
                int c = (cx * g.nc[1] + cy) * g.nc[2] + cz;
                for (int64_t e = cell_start[c] + threadIdx.x; e < cell_start[c + 1];
                     e += ROW_THREADS) {
                    int j = cell_atoms[e];
                    if (j == i || min_image_d2(pos, g.box, i, j) < r2) {
                        if (FILL) {
                            int s = atomicAdd(&count, 1);
                            if (s < CQ_ROW_CAP) buf[s] = j;
                        } else {
                            ++local;
                        }
                    }
                }
            }
    if (!FILL) {
        // deterministic: integer sums
        atomicAdd(&count, local);
        __syncthreads();
        if (threadIdx.x == 0) {
            row_count[i] = count;
            if (count > CQ_ROW_CAP) atomicOr(flag, 2);
        }
        return;
    }
    __syncthreads();
    const int m = count < CQ_ROW_CAP ? count : CQ_ROW_CAP;
    int p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (int t = m + threadIdx.x; t < p2; t += ROW_THREADS) buf[t] = 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < p2; t += ROW_THREADS) {
                int o = t ^ jj;
                if (o > t) {
                    int a = buf[t], b = buf[o];
                    bool up = (t & k) == 0;
                    if ((a > b) == up) {
                        buf[t] = b;
                        buf[o] = a;
                    }
                }
            }
            __syncthreads();
        }
    const int64_t base = row_ptr[i];
    for (int t = threadIdx.x; t < m; t += ROW_THREADS) col[base + t] = buf[t];
}

__global__ void k_block_rows(int n, const int64_t *row_ptr, int32_t *row)
{
    const int i = blockIdx.x;
    for (int64_t b = row_ptr[i] + threadIdx.x; b < row_ptr[i + 1]; b += blockDim.x) row[b] = i;
}

__global__ void k_block_sizes(int64_t nblk, const int32_t *row, const int32_t *col,
                              const int32_t *nb, int pad, int64_t *size)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    int64_t s = (int64_t)nb[row[b]] * nb[col[b]];
    size[b] = pad ? (s + 1) & ~int64_t(1) : s;
}

__device__ __forceinline__ int64_t find_in_row(const int64_t *rp, const int32_t *col, int i,
                                               int j)
{
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < rp[i + 1] && col[lo] == j) ? lo : -1;
}

__global__ void k_transpose(int64_t nblk, const int64_t *rp, const int32_t *row,
                            const int32_t *col, int64_t *tr)
{
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    tr[b] = find_in_row(rp, col, col[b], row[b]);
}

// Scatter of a coordinate list of blocks into pattern storage.
__global__ void k_scatter(int64_t n_pairs, const int32_t *pi, const int32_t *pj,
                          const int64_t *poff, const double *pv, const int32_t *nb,
                          const int64_t *rp, const int32_t *col, const int64_t *val_off,
                          double *out, int32_t *flag)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= n_pairs) return;
    const int i = pi[b], j = pj[b];
    const int64_t dst = find_in_row(rp, col, i, j);
    if (dst < 0) {
        if (lane == 0) atomicOr(flag, 4);
        return;
    }
    const int64_t sz = (int64_t)nb[i] * nb[j];
    if (poff[b + 1] - poff[b] != sz) {
        if (lane == 0) atomicOr(flag, 8);
        return;
    }
    for (int64_t e = lane; e < sz; e += 32) out[val_off[dst] + e] = pv[poff[b] + e];
}

// Batches: one CTA per atom row scans the atoms of the row's own cell in ascending order
// with that cell's box and range; a ballot per warp and a CTA prefix keep the output in
// ascending column order without sorting.
template <bool FILL>
__global__ void __launch_bounds__(ROW_THREADS)
k_rows_cellwise(const double *pos, const int32_t *cell_of, const int32_t *cell_start,
                const double *boxes, const double *r2s, int64_t *row_count,
                const int64_t *row_ptr, int32_t *col)
{
    __shared__ int wcount[ROW_THREADS / 32];
    const int i = blockIdx.x, c = cell_of[i];
    const int j0 = cell_start[c], j1 = cell_start[c + 1];
    const double r2 = r2s[c];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t run = FILL ? row_ptr[i] : 0;
    for (int base = j0; base < j1; base += ROW_THREADS) {
        const int j = base + threadIdx.x;
        const bool hit = j < j1 && (j == i || min_image_d2(pos, boxes + 3 * c, i, j) < r2);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcount[wid] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < ROW_THREADS / 32; ++w) {
            before += w < wid ? wcount[w] : 0;
            total += wcount[w];
        }
        if (FILL && hit) col[run + before + __popc(m & ((1u << lane) - 1u))] = j;
        run += total;
        __syncthreads();
    }
    if (!FILL && threadIdx.x == 0) row_count[i] = run;
}

}  // namespace

bool cq_same_atoms(const cq_pattern *a, const cq_pattern *b)
{
    if (a->geo == b->geo) return true;
    const Geometry &ga = *a->geo, &gb = *b->geo;
    if (ga.n_atoms != gb.n_atoms) return false;
    if (std::memcmp(ga.box, gb.box, sizeof(ga.box)) != 0) return false;
    if (ga.nb_host != gb.nb_host) return false;
    if (ga.cell_start != gb.cell_start || ga.boxes != gb.boxes) return false;
    return std::memcmp(ga.pos_host.data(), gb.pos_host.data(),
                       sizeof(double) * ga.pos_host.size()) == 0;
}

// Row counts (COUNT) or sorted columns (FILL) of a batch pattern.
static cq_status batch_rows(cq_ctx *ctx, const cq_pattern *p, bool fill, int64_t *row_count)
{
    const Geometry &g = *p->geo;
    void *v_r2;
    cq_status st = cq_scratch(ctx, "pb_r2", sizeof(double) * g.n_cells, &v_r2);
    if (st != CQ_OK) return st;
    std::vector<double> r2(g.n_cells);
    for (int c = 0; c < g.n_cells; ++c) r2[c] = p->ranges[c] * p->ranges[c];
    cudaMemcpyAsync(v_r2, r2.data(), sizeof(double) * g.n_cells, cudaMemcpyHostToDevice,
                    ctx->stream);
    const int n = g.n_atoms;
    if (fill)
        k_rows_cellwise<true><<<n, ROW_THREADS, 0, ctx->stream>>>(
            g.pos.as<double>(), g.cell_of.as<int32_t>(), g.cell_start_dev.as<int32_t>(),
            g.boxes_dev.as<double>(), (double *)v_r2, nullptr, p->row_ptr.as<int64_t>(),
            p->col.as<int32_t>());
    else
        k_rows_cellwise<false><<<n, ROW_THREADS, 0, ctx->stream>>>(
            g.pos.as<double>(), g.cell_of.as<int32_t>(), g.cell_start_dev.as<int32_t>(),
            g.boxes_dev.as<double>(), (double *)v_r2, row_count, nullptr, nullptr);
    cq_count_launch();
    st = cq_check_cuda(ctx, cudaGetLastError(), "batch pattern rows");
    if (st == CQ_OK)
        st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "batch pattern rows");
    return st;
}

cq_status cq_pattern_build_geo(cq_ctx *ctx, std::shared_ptr<Geometry> geo,
                               const std::vector<double> &ranges, cq_pattern **out)
{
    const int n = geo->n_atoms;
    cudaStream_t s = ctx->stream;
    const bool batch = geo->n_cells > 1;
    const double range = ranges[0];
    CellGrid g;
    int64_t ncell = 1;
    for (int c = 0; c < 3; ++c) {
        g.box[c] = geo->box[c];
        double q = range > 0.0 ? std::floor(geo->box[c] / range) : 64.0;
        int nc = (q >= 3.0 && !batch) ? (int)std::min(q, 64.0) : 1;
        g.nc[c] = nc;
        ncell *= nc;
    }
    std::unique_ptr<cq_pattern> p(new cq_pattern());
    p->ctx = ctx;
    p->id = ctx->next_id++;
    p->geo = geo;
    p->range = range;
    p->ranges = ranges;
    cq_status st;
    void *v_cell_of, *v_cell_cnt, *v_cell_start, *v_cursor, *v_cell_atoms, *v_rowcnt;
    if ((st = cq_scratch(ctx, "pb_cell_of", sizeof(int32_t) * n, &v_cell_of)) != CQ_OK ||
        (st = cq_scratch(ctx, "pb_cell_cnt", sizeof(int64_t) * ncell, &v_cell_cnt)) != CQ_OK ||
        (st = cq_scratch(ctx, "pb_cell_start", sizeof(int64_t) * (ncell + 1), &v_cell_start)) != CQ_OK ||
        (st = cq_scratch(ctx, "pb_cursor", sizeof(int64_t) * ncell, &v_cursor)) != CQ_OK ||
        (st = cq_scratch(ctx, "pb_cell_atoms", sizeof(int32_t) * n, &v_cell_atoms)) != CQ_OK ||
        (st = cq_scratch(ctx, "pb_rowcnt", sizeof(int64_t) * n, &v_rowcnt)) != CQ_OK)
        return st;
    cudaMemsetAsync(v_cell_cnt, 0, sizeof(int64_t) * ncell, s);
    cudaMemsetAsync(v_cursor, 0, sizeof(int64_t) * ncell, s);
    const double *pos = geo->pos.as<double>();
    k_cell_of<<<(n + 255) / 256, 256, 0, s>>>(n, pos, g, (int32_t *)v_cell_of,
                                              (int64_t *)v_cell_cnt);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)v_cell_cnt, (int64_t *)v_cell_start, ncell)) != CQ_OK)
        return st;
    k_cell_fill<<<(n + 255) / 256, 256, 0, s>>>(n, (int32_t *)v_cell_of,
                                                (int64_t *)v_cell_start, (int64_t *)v_cursor,
                                                (int32_t *)v_cell_atoms);
    cq_count_launch();
    const double r2 = range * range;
    if (batch) {
        if ((st = batch_rows(ctx, p.get(), false, (int64_t *)v_rowcnt)) != CQ_OK) return st;
    } else {
        k_rows<false><<<n, ROW_THREADS, 0, s>>>(n, pos, g, (int32_t *)v_cell_of,
                                                (int64_t *)v_cell_start, (int32_t *)v_cell_atoms,
                                                r2, (int64_t *)v_rowcnt, nullptr, nullptr,
                                                ctx->flag.as<int32_t>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "pattern rows")) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, p->row_ptr, sizeof(int64_t) * (n + 1))) != CQ_OK) return st;
    if ((st = cq_scan_i64(ctx, (int64_t *)v_rowcnt, p->row_ptr.as<int64_t>(), n)) != CQ_OK)
        return st;
    int32_t flag = 0;
    if ((st = cq_read_flag(ctx, &flag)) != CQ_OK) return st;
    if (flag & 2)
        return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: a row holds more than 8192 blocks");
    p->row_ptr_host.resize(n + 1);
    cudaMemcpyAsync(p->row_ptr_host.data(), p->row_ptr.ptr, sizeof(int64_t) * (n + 1),
                    cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "sync")) != CQ_OK) return st;
    p->n_blocks = p->row_ptr_host[n];
    for (int i = 0; i < n; ++i)
        p->max_row = std::max(p->max_row, p->row_ptr_host[i + 1] - p->row_ptr_host[i]);
    const int64_t nblk = p->n_blocks;
    if (nblk >= (int64_t(1) << 31))
        return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: more than 2^31 blocks");
    if ((st = cq_alloc(ctx, p->col, sizeof(int32_t) * nblk)) != CQ_OK ||
        (st = cq_alloc(ctx, p->row, sizeof(int32_t) * nblk)) != CQ_OK ||
        (st = cq_alloc(ctx, p->val_off, sizeof(int64_t) * (nblk + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, p->transpose, sizeof(int64_t) * nblk)) != CQ_OK)
        return st;
    if (batch) {
        if ((st = batch_rows(ctx, p.get(), true, nullptr)) != CQ_OK) return st;
    } else {
        k_rows<true><<<n, ROW_THREADS, 0, s>>>(n, pos, g, (int32_t *)v_cell_of,
                                               (int64_t *)v_cell_start, (int32_t *)v_cell_atoms,
                                               r2, nullptr, p->row_ptr.as<int64_t>(),
                                               p->col.as<int32_t>(), ctx->flag.as<int32_t>());
        cq_count_launch();
    }
    k_block_rows<<<n, 128, 0, s>>>(n, p->row_ptr.as<int64_t>(), p->row.as<int32_t>());
    cq_count_launch();
    void *v_sizes;
    if ((st = cq_scratch(ctx, "pb_sizes", sizeof(int64_t) * nblk, &v_sizes)) != CQ_OK) return st;
    const unsigned gb = (unsigned)((nblk + 255) / 256);
    void *v_scan;
    if ((st = cq_scratch(ctx, "pb_scan", sizeof(int64_t) * (nblk + 1), &v_scan)) != CQ_OK)
        return st;
    // unpadded total first (scalar count), then the padded offsets
    k_block_sizes<<<gb, 256, 0, s>>>(nblk, p->row.as<int32_t>(), p->col.as<int32_t>(),
                                     geo->nb.as<int32_t>(), 0, (int64_t *)v_sizes);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)v_sizes, (int64_t *)v_scan, nblk)) != CQ_OK)
        return st;
    cudaMemcpyAsync(&p->n_scalars, (int64_t *)v_scan + nblk, sizeof(int64_t),
                    cudaMemcpyDeviceToHost, s);
    k_block_sizes<<<gb, 256, 0, s>>>(nblk, p->row.as<int32_t>(), p->col.as<int32_t>(),
                                     geo->nb.as<int32_t>(), 1, (int64_t *)v_sizes);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)v_sizes, p->val_off.as<int64_t>(), nblk)) != CQ_OK)
        return st;
    k_transpose<<<gb, 256, 0, s>>>(nblk, p->row_ptr.as<int64_t>(), p->row.as<int32_t>(),
                                   p->col.as<int32_t>(), p->transpose.as<int64_t>());
    cq_count_launch();
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "pattern")) != CQ_OK) return st;
    int64_t nv = 0;
    cudaMemcpyAsync(&nv, p->val_off.as<int64_t>() + nblk, sizeof(int64_t),
                    cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "sync")) != CQ_OK) return st;
    p->n_values = nv;
    p->uniform = geo->uniform_nb ? (int)cq_pad2((int64_t)geo->uniform_nb * geo->uniform_nb) : 0;
    // per-cell segments: blocks of cell c are those of its atom rows
    const int nc = geo->n_cells;
    p->seg_blk.resize(nc + 1);
    p->seg_val.resize(nc + 1);
    p->seg_scalars.assign(nc, 0);
    for (int c = 0; c <= nc; ++c) p->seg_blk[c] = p->row_ptr_host[geo->cell_start[c]];
    for (int c = 0; c <= nc; ++c) {
        if (p->seg_blk[c] == nblk) {
            p->seg_val[c] = nv;
        } else {
            cudaMemcpyAsync(&p->seg_val[c], p->val_off.as<int64_t>() + p->seg_blk[c],
                            sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        }
    }
    if (nc > 1) {
        std::vector<int64_t> scal(nblk + 1);
        cudaMemcpyAsync(scal.data(), v_scan, sizeof(int64_t) * (nblk + 1),
                        cudaMemcpyDeviceToHost, s);
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "sync")) != CQ_OK) return st;
        for (int c = 0; c < nc; ++c) p->seg_scalars[c] = scal[p->seg_blk[c + 1]] - scal[p->seg_blk[c]];
    } else {
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "sync")) != CQ_OK) return st;
        p->seg_scalars[0] = p->n_scalars;
    }
    if ((st = cq_alloc(ctx, p->seg_blk_dev, sizeof(int64_t) * (nc + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, p->seg_val_dev, sizeof(int64_t) * (nc + 1))) != CQ_OK)
        return st;
    cudaMemcpyAsync(p->seg_blk_dev.ptr, p->seg_blk.data(), sizeof(int64_t) * (nc + 1),
                    cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->seg_val_dev.ptr, p->seg_val.data(), sizeof(int64_t) * (nc + 1),
                    cudaMemcpyHostToDevice, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "sync")) != CQ_OK) return st;
    *out = p.release();
    return CQ_OK;
}

cq_status cq_pattern_derived(cq_ctx *ctx, const cq_pattern *base, double ca,
                             const cq_pattern *pa, double cb, const cq_pattern *pb,
                             cq_pattern **out)
{
    std::vector<double> ranges(base->n_cells());
    for (int c = 0; c < base->n_cells(); ++c) ranges[c] = ca * pa->ranges[c] + cb * pb->ranges[c];
    auto key = std::make_pair(base->geo->id, ranges);
    auto it = ctx->derived.find(key);
    if (it != ctx->derived.end()) {
        *out = it->second;
        return CQ_OK;
    }
    cq_pattern *p = nullptr;
    cq_status st = cq_pattern_build_geo(ctx, base->geo, ranges, &p);
    if (st != CQ_OK) return st;
    p->owned_by_ctx = true;
    ctx->derived[key] = p;
    *out = p;
    return CQ_OK;
}

extern "C" cq_status cq_pattern_scatter(cq_ctx *ctx, const cq_pattern *p, int64_t n_pairs,
                                        const int32_t *pair_i_dev, const int32_t *pair_j_dev,
                                        const int64_t *pair_off_dev,
                                        const double *pair_values_dev, double *out)
{
    if (!ctx || !p || n_pairs < 0) return CQ_ERR_INVALID;
    if (p->ctx != ctx) return cq_fail(ctx, CQ_ERR_PATTERN, "pattern of another context");
    if (!out && p->n_values) return cq_fail(ctx, CQ_ERR_INVALID, "scatter: null output");
    if (n_pairs > 0 && (!pair_i_dev || !pair_j_dev || !pair_off_dev || !pair_values_dev))
        return cq_fail(ctx, CQ_ERR_INVALID, "scatter: null pair array");
    cq_status st = cq_check_cuda(ctx, cudaMemsetAsync(out, 0, sizeof(double) * p->n_values,
                                                      ctx->stream), "scatter");
    if (st != CQ_OK) return st;
    if (n_pairs > 0) {
        const unsigned grid = (unsigned)((n_pairs + 7) / 8);
        k_scatter<<<grid, 256, 0, ctx->stream>>>(n_pairs, pair_i_dev, pair_j_dev, pair_off_dev,
                                                 pair_values_dev, p->geo->nb.as<int32_t>(),
                                                 p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
                                                 p->val_off.as<int64_t>(), out,
                                                 ctx->flag.as<int32_t>());
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "scatter")) != CQ_OK) return st;
    }
    int32_t flag = 0;
    if ((st = cq_read_flag(ctx, &flag)) != CQ_OK) return st;
    if (flag & 4) return cq_fail(ctx, CQ_ERR_PATTERN, "scatter: a pair lies outside the pattern");
    if (flag & 8) return cq_fail(ctx, CQ_ERR_INVALID, "scatter: pair size differs from nb[i]*nb[j]");
    return CQ_OK;
}
