// Traces, inner products, norms, Gershgorin bounds (deterministic FP64 two-level
// reductions) and the elementwise kernels on pattern values.
//
// Reductions: stage 1 runs a fixed grid of RED_G CTAs; every thread accumulates its
// grid-stride share in a fixed order, each CTA combines its threads by a fixed tree into one
// partial; stage 2 (one CTA) combines the RED_G partials by a fixed tree.  The result does
// not depend on scheduling, so repeated runs are bitwise identical.  Padding values at the
// end of odd-sized blocks are never read.
#include <cfloat>

#include "cq_internal.cuh"

namespace {

constexpr int RED_G = 1024;
constexpr int RED_T = 256;

enum Op { SUM = 0, MIN = 1, MAX = 2 };

template <int OP>
__device__ __forceinline__ double combine(double a, double b)
{
    if (OP == SUM) return a + b;
    if (OP == MIN) return fmin(a, b);
    return fmax(a, b);
}

template <int OP>
__device__ __forceinline__ double identity_of()
{
    return OP == SUM ? 0.0 : (OP == MIN ? DBL_MAX : -DBL_MAX);
}

// Fixed-shape CTA tree over RED_T values; result valid in thread 0.
template <int OP>
__device__ double cta_reduce(double v)
{
    __shared__ double sh[RED_T / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = combine<OP>(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < RED_T / 32 ? sh[lane] : identity_of<OP>();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = combine<OP>(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// Stage 2: one CTA of RED_T threads folds `n` partials (strided by `stride`) into out.
template <int OP>
__global__ void k_final(const double *part, int n, int stride, double *out)
{
    double v = identity_of<OP>();
    for (int e = threadIdx.x; e < n; e += RED_T) v = combine<OP>(v, part[(int64_t)e * stride]);
    v = cta_reduce<OP>(v);
    if (threadIdx.x == 0) *out = v;
}

// Tr(A.B): warp per A block (i, j); B block (j, i) index from bmap (-1: absent).
__global__ void __launch_bounds__(RED_T)
k_trace(int64_t nblk, const int32_t *row, const int32_t *col, const int32_t *nb,
        const int64_t *a_off, const int64_t *b_off, const int64_t *bmap, const double *A,
        const double *B, double *part)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5);
    double s = 0.0;
    for (int64_t b = w0; b < nblk; b += (int64_t)RED_G * (RED_T / 32)) {
        const int64_t t = bmap[b];
        if (t < 0) continue;
        const int ni = nb[row[b]], nj = nb[col[b]];
        const double *a = A + a_off[b];
        const double *bb = B + b_off[t];
        for (int e = lane; e < ni * nj; e += 32) {
            const int r = e / nj, q = e - r * nj;
            s = fma(a[e], bb[q * ni + r], s);
        }
    }
    s = cta_reduce<SUM>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// <A, B> over the blocks of one pattern (padding skipped).
__global__ void __launch_bounds__(RED_T)
k_dot(int64_t nblk, const int32_t *row, const int32_t *col, const int32_t *nb,
      const int64_t *off, const double *A, const double *B, double *part)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5);
    double s = 0.0;
    for (int64_t b = w0; b < nblk; b += (int64_t)RED_G * (RED_T / 32)) {
        const int sz = nb[row[b]] * nb[col[b]];
        const int64_t o = off[b];
        for (int e = lane; e < sz; e += 32) s = fma(A[o + e], B[o + e], s);
    }
    s = cta_reduce<SUM>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_T)
k_frob2_mi(int64_t nblk, const int32_t *row, const int32_t *col, const int32_t *nb,
           const int64_t *off, const double *M, double *part)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5);
    double s = 0.0;
    for (int64_t b = w0; b < nblk; b += (int64_t)RED_G * (RED_T / 32)) {
        const int i = row[b], j = col[b];
        const int ni = nb[i], nj = nb[j];
        const int64_t o = off[b];
        for (int e = lane; e < ni * nj; e += 32) {
            double v = M[o + e];
            if (i == j && (e / nj) == (e % nj)) v -= 1.0;
            s = fma(v, v, s);
        }
    }
    s = cta_reduce<SUM>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Gershgorin data per scalar row: warp per atom row, lane r < n_i owns scalar row r.
__global__ void __launch_bounds__(RED_T)
k_row_bounds(int n_atoms, const int64_t *rp, const int32_t *col, const int32_t *nb,
             const int64_t *off, const double *M, double *part)
{
    const int lane = threadIdx.x & 31;
    const int w0 = blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5);
    double lo = DBL_MAX, hi = -DBL_MAX, amax = 0.0;
    for (int i = w0; i < n_atoms; i += RED_G * (RED_T / 32)) {
        const int ni = nb[i];
        if (lane >= ni) continue;
        double centre = 0.0, rad = 0.0, tot = 0.0;
        for (int64_t b = rp[i]; b < rp[i + 1]; ++b) {
            const int j = col[b], nj = nb[j];
            const double *m = M + off[b] + (int64_t)lane * nj;
            for (int q = 0; q < nj; ++q) {
                const double v = m[q];
                tot += fabs(v);
                if (j == i && q == lane)
                    centre = v;
                else
                    rad += fabs(v);
            }
        }
        lo = fmin(lo, centre - rad);
        hi = fmax(hi, centre + rad);
        amax = fmax(amax, tot);
    }
    lo = cta_reduce<MIN>(lo);
    hi = cta_reduce<MAX>(hi);
    amax = cta_reduce<MAX>(amax);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = lo;
        part[3 * blockIdx.x + 1] = hi;
        part[3 * blockIdx.x + 2] = amax;
    }
}

__global__ void k_axpby(int64_t n, double a, const double *x, double b, double *y)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (b == 0.0) ? a * x[e] : a * x[e] + b * y[e];
}

// dst_b = s * (src_ij or src_ji^T) + bb * dst_b; warp per destination block.
__global__ void k_gather(int64_t nblk, const int32_t *row, const int32_t *col,
                         const int32_t *nb, const int64_t *d_off, const int64_t *s_off,
                         const int64_t *map, int transpose, const double *src, double *dst,
                         double s, double bb)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int ni = nb[row[b]], nj = nb[col[b]];
    const int64_t m = map[b];
    double *d = dst + d_off[b];
    for (int e = lane; e < ni * nj; e += 32) {
        double v = 0.0;
        if (m >= 0) {
            const int r = e / nj, q = e - r * nj;
            v = transpose ? src[s_off[m] + q * ni + r] : src[s_off[m] + e];
        }
        d[e] = (bb == 0.0) ? s * v : s * v + bb * d[e];
    }
}

__global__ void k_identity(int n_atoms, const int64_t *rp, const int32_t *col,
                           const int32_t *nb, const int64_t *off, double *M, double s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_atoms) return;
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < i)
            lo = mid + 1;
        else
            hi = mid;
    }
    const int ni = nb[i];
    for (int r = 0; r < ni; ++r) M[off[lo] + r * ni + r] = s;
}

// G_E = 2[3(Z + Z^T) - 2((R1 + R1^T) + R2)], G_N = 12(U - R3) on P_L (warp per L block).
__global__ void k_lnv_grad(int64_t nblk, const int32_t *row, const int32_t *col,
                           const int32_t *nb, const int64_t *l_off, const int64_t *l_tr,
                           const int64_t *u_off, const int64_t *map_u, const int64_t *map_ut,
                           const double *Z, const double *U, const double *R1,
                           const double *R2, const double *R3, double *GE, double *GN)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int ni = nb[row[b]], nj = nb[col[b]];
    const int64_t lb = l_off[b], lt = l_off[l_tr[b]];
    const int64_t zb = map_u[b], zt = map_ut[b];
    for (int e = lane; e < ni * nj; e += 32) {
        const int r = e / nj, q = e - r * nj;
        const double z = zb >= 0 ? Z[u_off[zb] + e] : 0.0;
        const double zT = zt >= 0 ? Z[u_off[zt] + q * ni + r] : 0.0;
        const double u = zb >= 0 ? U[u_off[zb] + e] : 0.0;
        const double t = (R1[lb + e] + R1[lt + q * ni + r]) + R2[lb + e];
        GE[lb + e] = 2.0 * (3.0 * (z + zT) - 2.0 * t);
        GN[lb + e] = 12.0 * (u - R3[lb + e]);
    }
}

__global__ void k_lnv_grad_n(int64_t nblk, const int32_t *row, const int32_t *col,
                             const int32_t *nb, const int64_t *l_off, const int64_t *u_off,
                             const int64_t *map_u, const double *U, const double *R3,
                             double *GN)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int sz = nb[row[b]] * nb[col[b]];
    const int64_t lb = l_off[b], zb = map_u[b];
    for (int e = lane; e < sz; e += 32) {
        const double u = zb >= 0 ? U[u_off[zb] + e] : 0.0;
        GN[lb + e] = 12.0 * (u - R3[lb + e]);
    }
}

__global__ void k_lnv_grad_e(int64_t nblk, const int32_t *row, const int32_t *col,
                             const int32_t *nb, const int64_t *l_off, const int64_t *l_tr,
                             const int64_t *u_off, const int64_t *map_u, const int64_t *map_ut,
                             const double *Z, const double *R1, const double *R2, double *GE)
{
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    const int ni = nb[row[b]], nj = nb[col[b]];
    const int64_t lb = l_off[b], lt = l_off[l_tr[b]];
    const int64_t zb = map_u[b], zt = map_ut[b];
    for (int e = lane; e < ni * nj; e += 32) {
        const int r = e / nj, q = e - r * nj;
        const double z = zb >= 0 ? Z[u_off[zb] + e] : 0.0;
        const double zT = zt >= 0 ? Z[u_off[zt] + q * ni + r] : 0.0;
        const double t = (R1[lb + e] + R1[lt + q * ni + r]) + R2[lb + e];
        GE[lb + e] = 2.0 * (3.0 * (z + zT) - 2.0 * t);
    }
}

// ---------------- per-cell (segmented) versions: blockIdx.y = cell, RED_S CTAs per cell
constexpr int RED_S = 64;

__global__ void __launch_bounds__(RED_T)
k_trace_seg(const int64_t *seg, const int32_t *row, const int32_t *col, const int32_t *nb,
            const int64_t *a_off, const int64_t *b_off, const int64_t *bmap, const double *A,
            const double *B, double *part)
{
    const int lane = threadIdx.x & 31, c = blockIdx.y;
    const int64_t b0 = seg[c], b1 = seg[c + 1];
    double s = 0.0;
    for (int64_t b = b0 + (int64_t)blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5); b < b1;
         b += (int64_t)RED_S * (RED_T / 32)) {
        const int64_t t = bmap[b];
        if (t < 0) continue;
        const int ni = nb[row[b]], nj = nb[col[b]];
        const double *a = A + a_off[b];
        const double *bb = B + b_off[t];
        for (int e = lane; e < ni * nj; e += 32) {
            const int r = e / nj, q = e - r * nj;
            s = fma(a[e], bb[q * ni + r], s);
        }
    }
    s = cta_reduce<SUM>(s);
    if (threadIdx.x == 0) part[(int64_t)c * RED_S + blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_T)
k_dot_seg(const int64_t *seg, const int32_t *row, const int32_t *col, const int32_t *nb,
          const int64_t *off, const double *A, const double *B, double *part)
{
    const int lane = threadIdx.x & 31, c = blockIdx.y;
    const int64_t b0 = seg[c], b1 = seg[c + 1];
    double s = 0.0;
    for (int64_t b = b0 + (int64_t)blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5); b < b1;
         b += (int64_t)RED_S * (RED_T / 32)) {
        const int sz = nb[row[b]] * nb[col[b]];
        const int64_t o = off[b];
        for (int e = lane; e < sz; e += 32) s = fma(A[o + e], B[o + e], s);
    }
    s = cta_reduce<SUM>(s);
    if (threadIdx.x == 0) part[(int64_t)c * RED_S + blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_T)
k_row_bounds_seg(const int32_t *cell_start, const int64_t *rp, const int32_t *col,
                 const int32_t *nb, const int64_t *off, const double *M, double *part)
{
    const int lane = threadIdx.x & 31, c = blockIdx.y;
    double lo = DBL_MAX, hi = -DBL_MAX, amax = 0.0;
    for (int i = cell_start[c] + blockIdx.x * (RED_T / 32) + (threadIdx.x >> 5);
         i < cell_start[c + 1]; i += RED_S * (RED_T / 32)) {
        const int ni = nb[i];
        if (lane >= ni) continue;
        double centre = 0.0, rad = 0.0, tot = 0.0;
        for (int64_t b = rp[i]; b < rp[i + 1]; ++b) {
            const int j = col[b], nj = nb[j];
            const double *m = M + off[b] + (int64_t)lane * nj;
            for (int q = 0; q < nj; ++q) {
                const double v = m[q];
                tot += fabs(v);
                if (j == i && q == lane)
                    centre = v;
                else
                    rad += fabs(v);
            }
        }
        lo = fmin(lo, centre - rad);
        hi = fmax(hi, centre + rad);
        amax = fmax(amax, tot);
    }
    lo = cta_reduce<MIN>(lo);
    hi = cta_reduce<MAX>(hi);
    amax = cta_reduce<MAX>(amax);
    if (threadIdx.x == 0) {
        const int64_t k = (int64_t)c * RED_S + blockIdx.x;
        part[3 * k + 0] = lo;
        part[3 * k + 1] = hi;
        part[3 * k + 2] = amax;
    }
}

// one CTA per cell folds that cell's RED_S partials (strided) into out[cell * ostride]
template <int OP>
__global__ void k_final_seg(const double *part, int stride, double *out, int ostride)
{
    const int c = blockIdx.x;
    double v = identity_of<OP>();
    for (int e = threadIdx.x; e < RED_S; e += RED_T)
        v = combine<OP>(v, part[((int64_t)c * RED_S + e) * stride]);
    v = cta_reduce<OP>(v);
    if (threadIdx.x == 0) out[(int64_t)c * ostride] = v;
}

__global__ void k_axpby_seg(const int64_t *seg_val, const double *coef, int n_cells,
                            const double *x, double *y)
{
    const int c = blockIdx.y;
    const double a = coef[c], b = coef[n_cells + c];
    const int64_t v1 = seg_val[c + 1];
    for (int64_t e = seg_val[c] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < v1;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (b == 0.0) ? a * x[e] : a * x[e] + b * y[e];
}

__global__ void k_identity_seg(int n_atoms, const int32_t *cell_of, const int64_t *rp,
                               const int32_t *col, const int32_t *nb, const int64_t *off,
                               const double *scale, double *M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_atoms) return;
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < i)
            lo = mid + 1;
        else
            hi = mid;
    }
    const int ni = nb[i];
    const double s = scale[cell_of[i]];
    for (int r = 0; r < ni; ++r) M[off[lo] + r * ni + r] = s;
}

cq_status red_part(cq_ctx *ctx, double **part)
{
    void *p;
    cq_status st = cq_scratch(ctx, "red_part", sizeof(double) * 3 * RED_G, &p);
    *part = (double *)p;
    return st;
}

}  // namespace

cq_status cq_trace_dev(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                       const cq_pattern *pB, const double *B, int slot)
{
    const int64_t *bmap;
    cq_status st = cq_get_map(ctx, pB, pA, 1, &bmap);
    if (st != CQ_OK) return st;
    double *part;
    if ((st = red_part(ctx, &part)) != CQ_OK) return st;
    k_trace<<<RED_G, RED_T, 0, ctx->stream>>>(pA->n_blocks, pA->row.as<int32_t>(),
                                              pA->col.as<int32_t>(), pA->geo->nb.as<int32_t>(),
                                              pA->val_off.as<int64_t>(), pB->val_off.as<int64_t>(),
                                              bmap, A, B, part);
    k_final<SUM><<<1, RED_T, 0, ctx->stream>>>(part, RED_G, 1, ctx->red_out.as<double>() + slot);
    cq_count_launch(2);
    return cq_check_cuda(ctx, cudaGetLastError(), "trace");
}

cq_status cq_dot_dev(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                     int slot)
{
    double *part;
    cq_status st = red_part(ctx, &part);
    if (st != CQ_OK) return st;
    k_dot<<<RED_G, RED_T, 0, ctx->stream>>>(p->n_blocks, p->row.as<int32_t>(),
                                            p->col.as<int32_t>(), p->geo->nb.as<int32_t>(),
                                            p->val_off.as<int64_t>(), A, B, part);
    k_final<SUM><<<1, RED_T, 0, ctx->stream>>>(part, RED_G, 1, ctx->red_out.as<double>() + slot);
    cq_count_launch(2);
    return cq_check_cuda(ctx, cudaGetLastError(), "dot");
}

cq_status cq_frob2_minus_identity_dev(cq_ctx *ctx, const cq_pattern *p, const double *M,
                                      int slot)
{
    double *part;
    cq_status st = red_part(ctx, &part);
    if (st != CQ_OK) return st;
    k_frob2_mi<<<RED_G, RED_T, 0, ctx->stream>>>(p->n_blocks, p->row.as<int32_t>(),
                                                 p->col.as<int32_t>(), p->geo->nb.as<int32_t>(),
                                                 p->val_off.as<int64_t>(), M, part);
    k_final<SUM><<<1, RED_T, 0, ctx->stream>>>(part, RED_G, 1, ctx->red_out.as<double>() + slot);
    cq_count_launch(2);
    return cq_check_cuda(ctx, cudaGetLastError(), "frob2");
}

cq_status cq_row_bounds_dev(cq_ctx *ctx, const cq_pattern *p, const double *M, int slot)
{
    double *part;
    cq_status st = red_part(ctx, &part);
    if (st != CQ_OK) return st;
    k_row_bounds<<<RED_G, RED_T, 0, ctx->stream>>>(p->geo->n_atoms, p->row_ptr.as<int64_t>(),
                                                   p->col.as<int32_t>(), p->geo->nb.as<int32_t>(),
                                                   p->val_off.as<int64_t>(), M, part);
    double *o = ctx->red_out.as<double>() + slot;
    k_final<MIN><<<1, RED_T, 0, ctx->stream>>>(part + 0, RED_G, 3, o + 0);
    k_final<MAX><<<1, RED_T, 0, ctx->stream>>>(part + 1, RED_G, 3, o + 1);
    k_final<MAX><<<1, RED_T, 0, ctx->stream>>>(part + 2, RED_G, 3, o + 2);
    cq_count_launch(4);
    return cq_check_cuda(ctx, cudaGetLastError(), "row bounds");
}

cq_status cq_axpby(cq_ctx *ctx, int64_t n, double a, const double *x, double b, double *y)
{
    if (n == 0) return CQ_OK;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    if (blocks > cap) blocks = cap;
    k_axpby<<<(unsigned)blocks, 256, 0, ctx->stream>>>(n, a, x, b, y);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "axpby");
}

cq_status cq_gather(cq_ctx *ctx, const cq_pattern *pSrc, const double *src,
                    const cq_pattern *pDst, double *dst, int transpose, double s, double b)
{
    const int64_t *map;
    cq_status st = cq_get_map(ctx, pSrc, pDst, transpose, &map);
    if (st != CQ_OK) return st;
    if (pDst->n_blocks == 0) return CQ_OK;
    k_gather<<<(unsigned)((pDst->n_blocks + 7) / 8), 256, 0, ctx->stream>>>(
        pDst->n_blocks, pDst->row.as<int32_t>(), pDst->col.as<int32_t>(),
        pDst->geo->nb.as<int32_t>(), pDst->val_off.as<int64_t>(), pSrc->val_off.as<int64_t>(), map,
        transpose, src, dst, s, b);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "gather");
}

cq_status cq_set_identity(cq_ctx *ctx, const cq_pattern *p, double *M, double s)
{
    cq_status st = cq_check_cuda(ctx, cudaMemsetAsync(M, 0, sizeof(double) * p->n_values,
                                                      ctx->stream), "identity");
    if (st != CQ_OK) return st;
    const int n = p->geo->n_atoms;
    k_identity<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, p->row_ptr.as<int64_t>(),
                                                        p->col.as<int32_t>(),
                                                        p->geo->nb.as<int32_t>(),
                                                        p->val_off.as<int64_t>(), M, s);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "identity");
}

cq_status cq_lnv_gradients(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                           const double *Z, const double *U, const double *R1,
                           const double *R2, const double *R3, double *GE, double *GN)
{
    const int64_t *mu, *mut;
    cq_status st = cq_get_map(ctx, pU, pL, 0, &mu);
    if (st != CQ_OK) return st;
    if ((st = cq_get_map(ctx, pU, pL, 1, &mut)) != CQ_OK) return st;
    if (pL->n_blocks == 0) return CQ_OK;
    k_lnv_grad<<<(unsigned)((pL->n_blocks + 7) / 8), 256, 0, ctx->stream>>>(
        pL->n_blocks, pL->row.as<int32_t>(), pL->col.as<int32_t>(), pL->geo->nb.as<int32_t>(),
        pL->val_off.as<int64_t>(), pL->transpose.as<int64_t>(), pU->val_off.as<int64_t>(), mu, mut,
        Z, U, R1, R2, R3, GE, GN);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "lnv gradients");
}

// ---------------------------------------------------------------- per-cell host wrappers

static cq_status seg_part(cq_ctx *ctx, int n_cells, double **part)
{
    void *p;
    cq_status st = cq_scratch(ctx, "red_part_seg", sizeof(double) * 3 * RED_S * n_cells, &p);
    *part = (double *)p;
    return st;
}

cq_status cq_trace_seg_dev(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                           const cq_pattern *pB, const double *B, int slot)
{
    const int64_t *bmap;
    cq_status st = cq_get_map(ctx, pB, pA, 1, &bmap);
    if (st != CQ_OK) return st;
    const int nc = pA->n_cells();
    double *part;
    if ((st = seg_part(ctx, nc, &part)) != CQ_OK) return st;
    k_trace_seg<<<dim3(RED_S, nc), RED_T, 0, ctx->stream>>>(
        pA->seg_blk_dev.as<int64_t>(), pA->row.as<int32_t>(), pA->col.as<int32_t>(),
        pA->geo->nb.as<int32_t>(), pA->val_off.as<int64_t>(), pB->val_off.as<int64_t>(), bmap, A,
        B, part);
    k_final_seg<SUM><<<nc, RED_T, 0, ctx->stream>>>(part, 1, ctx->red_out.as<double>() + slot, 1);
    cq_count_launch(2);
    return cq_check_cuda(ctx, cudaGetLastError(), "trace (cells)");
}

cq_status cq_dot_seg_dev(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                         int slot)
{
    const int nc = p->n_cells();
    double *part;
    cq_status st = seg_part(ctx, nc, &part);
    if (st != CQ_OK) return st;
    k_dot_seg<<<dim3(RED_S, nc), RED_T, 0, ctx->stream>>>(
        p->seg_blk_dev.as<int64_t>(), p->row.as<int32_t>(), p->col.as<int32_t>(),
        p->geo->nb.as<int32_t>(), p->val_off.as<int64_t>(), A, B, part);
    k_final_seg<SUM><<<nc, RED_T, 0, ctx->stream>>>(part, 1, ctx->red_out.as<double>() + slot, 1);
    cq_count_launch(2);
    return cq_check_cuda(ctx, cudaGetLastError(), "dot (cells)");
}

cq_status cq_row_bounds_seg_dev(cq_ctx *ctx, const cq_pattern *p, const double *M, int slot)
{
    const int nc = p->n_cells();
    double *part;
    cq_status st = seg_part(ctx, nc, &part);
    if (st != CQ_OK) return st;
    k_row_bounds_seg<<<dim3(RED_S, nc), RED_T, 0, ctx->stream>>>(
        p->geo->cell_start_dev.as<int32_t>(), p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
        p->geo->nb.as<int32_t>(), p->val_off.as<int64_t>(), M, part);
    double *o = ctx->red_out.as<double>() + slot;
    k_final_seg<MIN><<<nc, RED_T, 0, ctx->stream>>>(part + 0, 3, o + 0, 3);
    k_final_seg<MAX><<<nc, RED_T, 0, ctx->stream>>>(part + 1, 3, o + 1, 3);
    k_final_seg<MAX><<<nc, RED_T, 0, ctx->stream>>>(part + 2, 3, o + 2, 3);
    cq_count_launch(4);
    return cq_check_cuda(ctx, cudaGetLastError(), "row bounds (cells)");
}

cq_status cq_axpby_seg(cq_ctx *ctx, const cq_pattern *p, const double *a, const double *x,
                       const double *b, double *y)
{
    const int nc = p->n_cells();
    void *v;
    cq_status st = cq_scratch(ctx, "seg_coef", sizeof(double) * 2 * nc, &v);
    if (st != CQ_OK) return st;
    std::vector<double> coef(a, a + nc);
    coef.insert(coef.end(), b, b + nc);
    cudaMemcpyAsync(v, coef.data(), sizeof(double) * 2 * nc, cudaMemcpyHostToDevice, ctx->stream);
    k_axpby_seg<<<dim3(64, nc), 256, 0, ctx->stream>>>(p->seg_val_dev.as<int64_t>(), (double *)v,
                                                       nc, x, y);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "axpby (cells)");
}

cq_status cq_set_identity_seg(cq_ctx *ctx, const cq_pattern *p, double *M, const double *s)
{
    const int nc = p->n_cells();
    cq_status st = cq_check_cuda(ctx, cudaMemsetAsync(M, 0, sizeof(double) * p->n_values,
                                                      ctx->stream), "identity");
    if (st != CQ_OK) return st;
    void *v;
    if ((st = cq_scratch(ctx, "seg_scale", sizeof(double) * nc, &v)) != CQ_OK) return st;
    cudaMemcpyAsync(v, s, sizeof(double) * nc, cudaMemcpyHostToDevice, ctx->stream);
    const int n = p->geo->n_atoms;
    k_identity_seg<<<(n + 127) / 128, 128, 0, ctx->stream>>>(
        n, p->geo->cell_of.as<int32_t>(), p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
        p->geo->nb.as<int32_t>(), p->val_off.as<int64_t>(), (const double *)v, M);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "identity (cells)");
}

cq_status cq_lnv_gradient_n(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                            const double *U, const double *R3, double *GN)
{
    const int64_t *mu;
    cq_status st = cq_get_map(ctx, pU, pL, 0, &mu);
    if (st != CQ_OK) return st;
    if (pL->n_blocks == 0) return CQ_OK;
    k_lnv_grad_n<<<(unsigned)((pL->n_blocks + 7) / 8), 256, 0, ctx->stream>>>(
        pL->n_blocks, pL->row.as<int32_t>(), pL->col.as<int32_t>(), pL->geo->nb.as<int32_t>(),
        pL->val_off.as<int64_t>(), pU->val_off.as<int64_t>(), mu, U, R3, GN);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "lnv gradient N");
}

cq_status cq_lnv_gradient_e(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                            const double *Z, const double *R1, const double *R2, double *GE)
{
    const int64_t *mu, *mut;
    cq_status st = cq_get_map(ctx, pU, pL, 0, &mu);
    if (st != CQ_OK) return st;
    if ((st = cq_get_map(ctx, pU, pL, 1, &mut)) != CQ_OK) return st;
    if (pL->n_blocks == 0) return CQ_OK;
    k_lnv_grad_e<<<(unsigned)((pL->n_blocks + 7) / 8), 256, 0, ctx->stream>>>(
        pL->n_blocks, pL->row.as<int32_t>(), pL->col.as<int32_t>(), pL->geo->nb.as<int32_t>(),
        pL->val_off.as<int64_t>(), pL->transpose.as<int64_t>(), pU->val_off.as<int64_t>(), mu,
        mut, Z, R1, R2, GE);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "lnv gradient E");
}
