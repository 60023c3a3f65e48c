// Learned initial guess for the density matrix L: a small MLP maps a descriptor of each atom
// pair's local environment to the pair's L block expressed in a pair frame; the block is
// rotated back to the global orbital frame.  Hand-written kernels: descriptors and frames,
// target extraction (global -> frame), MLP forward/backward (BF16 weights, FP32
// accumulation), Adam, and the apply step (frame -> global, both (i,j) and (j,i) blocks).
//
// Pair frame (i, j), i != j: e3 along r_j - r_i; e1 toward the atom nearest to the bond
// midpoint (other than i, j; ties: lowest index), made orthogonal to e3; e2 = e3 x e1.
// On-site (i, i): e3 toward i's nearest neighbour, e1 toward its second nearest.  Only
// blocks with i <= j are predicted; (j, i) is the transpose.  Uniform 9- or 4-orbital bases.
//
// Descriptor (64 numbers): 10 Gaussians of the pair distance (centres 1.6 p bohr, width
// 1.6) and, for the atoms k within 8 bohr of the midpoint m (k != i, j), sum_k h_n(|r_k - m|)
// Y_a(unit(r_k - m) in the pair frame) for 6 radial Gaussians h_n (centres 1.6 n, width
// 1.2, cosine cut at 8) and the 9 real harmonics Y_a up to l = 2.
#include <cuda_bf16.h>

#include <cmath>
#include <random>

#include "cq_internal.cuh"

#define CQ_TRY(x)                          \
    do {                                   \
        cq_status _st = (x);               \
        if (_st != CQ_OK) return _st;      \
    } while (0)

namespace {

constexpr int NDESC = 64;
constexpr int NOUT = 81;
constexpr float R_ENV = 8.0f;

struct Box3 {
    double v[3];
};

__device__ __forceinline__ void min_image(const double *pos, const Box3 &box, int i, int j,
                                          double d[3])
{
    for (int c = 0; c < 3; ++c) {
        double x = pos[3 * j + c] - pos[3 * i + c];
        d[c] = x - box.v[c] * rint(x / box.v[c]);
    }
}

__device__ __forceinline__ void normalize3(double v[3])
{
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int c = 0; c < 3; ++c) v[c] /= n;
}

// Real d orbitals as unit-Frobenius quadratic forms (xy, yz, zx, x2-y2, 3z2-r2).
__device__ void dform(int a, double q[3][3])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) q[r][c] = 0.0;
    const double h = 0.70710678118654752440, s6 = 0.40824829046386301637;
    switch (a) {
    case 0: q[0][1] = q[1][0] = h; break;
    case 1: q[1][2] = q[2][1] = h; break;
    case 2: q[2][0] = q[0][2] = h; break;
    case 3: q[0][0] = h; q[1][1] = -h; break;
    default: q[0][0] = q[1][1] = -s6; q[2][2] = 2.0 * s6; break;
    }
}

// Orbital rotation D (local <- global) for a frame with rows R = (e1, e2, e3):
// s -> 1, p -> R, d -> D2[a][b] = <Q_b, R^T Q_a R>_F.
__device__ void orbital_rotation(const double R[3][3], int nb, double D[9][9])
{
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) D[a][b] = 0.0;
    D[0][0] = 1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) D[1 + a][1 + b] = R[a][b];
    if (nb < 9) return;
    for (int a = 0; a < 5; ++a) {
        double qa[3][3], t[3][3];
        dform(a, qa);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v) acc += R[u][r] * qa[u][v] * R[v][c];
                t[r][c] = acc;
            }
        for (int b = 0; b < 5; ++b) {
            double qb[3][3];
            dform(b, qb);
            double acc = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) acc += qb[r][c] * t[r][c];
            D[4 + a][4 + b] = acc;
        }
    }
}

// Frame and descriptor of pair block b = (i, j), i <= j, from the atoms of row i of P_L.
__global__ void k_descriptors(int64_t n_pairs, const int32_t *pairs, const int32_t *row,
                              const int32_t *col, const int64_t *rp, const double *pos,
                              Box3 box, float *desc, float *frames)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int b = pairs[p];
    const int i = row[b], j = col[b];
    double dij[3] = {0.0, 0.0, 0.0};
    double e3[3], e1[3] = {0.0, 0.0, 0.0};
    double m[3];  // midpoint relative to atom i
    if (i != j) {
        min_image(pos, box, i, j, dij);
        for (int c = 0; c < 3; ++c) {
            e3[c] = dij[c];
            m[c] = 0.5 * dij[c];
        }
    } else {
        // nearest neighbour of i sets e3
        double best = 1e300;
        int kb = -1;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int k = col[e];
            if (k == i) continue;
            double d[3];
            min_image(pos, box, i, k, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < best || (r2 == best && k < kb)) {
                best = r2;
                kb = k;
                e3[0] = d[0];
                e3[1] = d[1];
                e3[2] = d[2];
            }
        }
        if (kb < 0) {
            e3[0] = 0.0;
            e3[1] = 0.0;
            e3[2] = 1.0;
        }
        m[0] = m[1] = m[2] = 0.0;
    }
    normalize3(e3);
    // third atom: nearest to the midpoint (other than i, j; for on-site, other than e3's)
    {
        double best = 1e300;
        int kb = -1;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int k = col[e];
            if (k == i || k == j) continue;
            double d[3];
            min_image(pos, box, i, k, d);
            double w[3] = {d[0] - m[0], d[1] - m[1], d[2] - m[2]};
            const double along = w[0] * e3[0] + w[1] * e3[1] + w[2] * e3[2];
            double perp[3] = {w[0] - along * e3[0], w[1] - along * e3[1], w[2] - along * e3[2]};
            const double pn = sqrt(perp[0] * perp[0] + perp[1] * perp[1] + perp[2] * perp[2]);
            if (pn < 1e-6) continue;  // on the axis: no azimuth
            const double r2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            if (r2 < best || (r2 == best && k < kb)) {
                best = r2;
                kb = k;
                for (int c = 0; c < 3; ++c) e1[c] = perp[c] / pn;
            }
        }
        if (kb < 0) {  // no off-axis atom: any perpendicular
            double h[3] = {fabs(e3[0]) < 0.9 ? 1.0 : 0.0, fabs(e3[0]) < 0.9 ? 0.0 : 1.0, 0.0};
            const double along = h[0] * e3[0] + h[1] * e3[1] + h[2] * e3[2];
            for (int c = 0; c < 3; ++c) e1[c] = h[c] - along * e3[c];
            normalize3(e1);
        }
    }
    double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                    e3[0] * e1[1] - e3[1] * e1[0]};
    float *fr = frames + p * 9;
    for (int c = 0; c < 3; ++c) {
        fr[c] = (float)e1[c];
        fr[3 + c] = (float)e2[c];
        fr[6 + c] = (float)e3[c];
    }
    float f[NDESC];
    for (int q = 0; q < NDESC; ++q) f[q] = 0.f;
    const float rij = (float)sqrt(dij[0] * dij[0] + dij[1] * dij[1] + dij[2] * dij[2]);
    for (int q = 0; q < 10; ++q) {
        const float x = (rij - 1.6f * q) / 1.6f;
        f[q] = __expf(-0.5f * x * x);
    }
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int k = col[e];
        if (k == i || k == j) continue;
        double d[3];
        min_image(pos, box, i, k, d);
        const double w[3] = {d[0] - m[0], d[1] - m[1], d[2] - m[2]};
        const float rho = (float)sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (rho >= R_ENV || rho < 1e-6f) continue;
        const float x = (float)((w[0] * e1[0] + w[1] * e1[1] + w[2] * e1[2]) / rho);
        const float y = (float)((w[0] * e2[0] + w[1] * e2[1] + w[2] * e2[2]) / rho);
        const float z = (float)((w[0] * e3[0] + w[1] * e3[1] + w[2] * e3[2]) / rho);
        const float ang[9] = {1.f, z, x, y, 0.5f * (3.f * z * z - 1.f), x * z, y * z,
                              0.5f * (x * x - y * y), x * y};
        const float fc = 0.5f * (1.f + __cosf(3.14159265f * rho / R_ENV));
        for (int n = 0; n < 6; ++n) {
            const float t = (rho - 1.6f * n) / 1.2f;
            const float h = __expf(-0.5f * t * t) * fc;
            for (int a = 0; a < 9; ++a) f[10 + 9 * n + a] += h * ang[a];
        }
    }
    float *o = desc + p * NDESC;
    for (int q = 0; q < NDESC; ++q) o[q] = f[q];
}

// targets: the (i, j) block of L in the pair frame, L_loc = D L D^T (row-major nb x nb,
// zero-padded to 81)
__global__ void k_targets(int64_t n_pairs, int nb, int stride, const int32_t *pairs,
                          const float *frames, const double *L, float *targets)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    double R[3][3], D[9][9], T[9][9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[r][c] = frames[p * 9 + 3 * r + c];
    orbital_rotation(R, nb, D);
    const double *blk = L + (int64_t)pairs[p] * stride;
    for (int a = 0; a < nb; ++a)
        for (int c = 0; c < nb; ++c) {
            double acc = 0.0;
            for (int u = 0; u < nb; ++u) acc += D[a][u] * blk[u * nb + c];
            T[a][c] = acc;
        }
    float *o = targets + p * NOUT;
    for (int a = 0; a < 9; ++a)
        for (int c = 0; c < 9; ++c) {
            double acc = 0.0;
            if (a < nb && c < nb)
                for (int v = 0; v < nb; ++v) acc += T[a][v] * D[c][v];
            o[a * 9 + c] = (float)acc;
        }
}

// apply: block (i, j) = D^T L_loc D and block (j, i) = its transpose
__global__ void k_apply(int64_t n_pairs, int nb, int stride, const int32_t *pairs,
                        const int64_t *tr, const float *frames, const float *pred,
                        const float *mean, const float *scale, double *L)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    double R[3][3], D[9][9], T[9][9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[r][c] = frames[p * 9 + 3 * r + c];
    orbital_rotation(R, nb, D);
    const float *y = pred + p * NOUT;
    double loc[9][9];
    for (int a = 0; a < 9; ++a)
        for (int c = 0; c < 9; ++c)
            loc[a][c] = (double)y[a * 9 + c] * scale[a * 9 + c] + mean[a * 9 + c];
    for (int a = 0; a < nb; ++a)
        for (int c = 0; c < nb; ++c) {
            double acc = 0.0;
            for (int u = 0; u < nb; ++u) acc += D[u][a] * loc[u][c];
            T[a][c] = acc;
        }
    const int b = pairs[p];
    double *blk = L + (int64_t)b * stride;
    double *blt = L + tr[b] * stride;
    for (int a = 0; a < nb; ++a)
        for (int c = 0; c < nb; ++c) {
            double acc = 0.0;
            for (int v = 0; v < nb; ++v) acc += T[a][v] * D[v][c];
            blk[a * nb + c] = acc;
            blt[c * nb + a] = acc;
        }
}

__global__ void k_pair_flags(int64_t nblk, const int32_t *row, const int32_t *col, int64_t *f)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblk) f[b] = row[b] <= col[b] ? 1 : 0;
}

__global__ void k_pair_fill(int64_t nblk, const int32_t *row, const int32_t *col,
                            const int64_t *pos, int32_t *pairs)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblk && row[b] <= col[b]) pairs[pos[b]] = (int32_t)b;
}

// ---------------------------------------------------------------- MLP kernels

// C[M x N] (+)= op(A) op(B) in FP32 with 64 x 64 tiles, 16 x 16 threads, 4 x 4 outputs each.
// A: FP32, op(A)[m][k] = TA ? A[k * lda + m] : A[m * lda + k];
// B: BT (float or bf16), op(B)[k][n] = TB ? B[n * ldb + k] : B[k * ldb + n].
// The K range [k0, k1) lets callers split a long reduction into deterministic partials.
template <bool TA, bool TB, typename BT>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, const float *A, int lda, const BT *B, int ldb, float *C, int ldc,
       int64_t k0, int64_t k1, int64_t c_stride_z, int64_t k_chunk)
{
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int64_t kb = k0 + (int64_t)blockIdx.z * k_chunk;
    const int64_t ke = min(k1, kb + k_chunk);
    float acc[4][4] = {};
    for (int64_t kt = kb; kt < ke; kt += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int64_t k = kt + kk;
            const int m = m0 + mm;
            float va = 0.f;
            if (k < ke && m < M) va = TA ? A[k * lda + m] : A[(int64_t)m * lda + k];
            As[kk][mm] = va;
            const int n = n0 + mm;
            float vb = 0.f;
            if (k < ke && n < N) vb = (float)(TB ? B[(int64_t)n * ldb + k] : B[k * ldb + n]);
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    float *Cz = C + (int64_t)blockIdx.z * c_stride_z;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int m = m0 + ty * 4 + r, n = n0 + tx * 4 + c;
            if (m < M && n < N) Cz[(int64_t)m * ldc + n] = acc[r][c];
        }
}

#include "mlp_tc.cuh"

// Z += bias; H = silu(Z) (hidden) or H = Z (output); Hb (if not null) = bf16(H)
__global__ void k_bias_act(int64_t M, int N, const float *bias, float *Z, float *H, int act,
                           __nv_bfloat16 *Hb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const float z = Z[e] + bias[e % N];
    Z[e] = z;
    const float h = act ? z / (1.f + __expf(-z)) : z;
    H[e] = h;
    if (Hb) Hb[e] = __float2bfloat16(h);
}

// dZ = dH * silu'(Z)
__global__ void k_act_back(int64_t n, const float *Z, const float *dH, float *dZ)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float z = Z[e], s = 1.f / (1.f + __expf(-z));
    dZ[e] = dH[e] * (s * (1.f + z * (1.f - s)));
}

// loss = mean (Y - T)^2 over n x 81 (per-CTA partials), dY = 2 (Y - T) / (n * 81)
__global__ void k_mse(int64_t n, const float *Y, const float *T, float *dY, float *part)
{
    __shared__ float sh[256];
    const int64_t tot = n * NOUT;
    float s = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[e] - T[e];
        s += d * d;
        dY[e] = 2.f * d / (float)tot;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// adds the 256 block partials of k_mse (fixed order) and the batch's row count to the
// running sums acc[0], acc[1] (one CTA of 256 threads)
__global__ void k_loss_accum(const float *part, int64_t rows, double *acc)
{
    __shared__ double sh[256];
    sh[threadIdx.x] = (double)part[threadIdx.x];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        acc[0] += sh[0];
        acc[1] += (double)rows;
    }
}

// sum of `parts` partial matrices (deterministic order) + column sums for bias gradients
__global__ void k_sum_parts(int64_t n, int parts, int64_t stride, const float *src, float *dst)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float s = 0.f;
    for (int q = 0; q < parts; ++q) s += src[q * stride + e];
    dst[e] = s;
}

__global__ void k_colsum(int64_t M, int N, const float *dZ, float *db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int64_t m = 0; m < M; ++m) s += dZ[m * N + n];
    db[n] = s;
}

// Adam on FP32 master weights; refresh the BF16 copy the forward pass reads.
__global__ void k_adam(int64_t n, float *w, const float *g, float *mo, float *ve,
                       __nv_bfloat16 *wb, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gr = g[e];
    const float m = b1 * mo[e] + (1.f - b1) * gr;
    const float v = b2 * ve[e] + (1.f - b2) * gr * gr;
    mo[e] = m;
    ve[e] = v;
    const float nw = w[e] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    w[e] = nw;
    if (wb) wb[e] = __float2bfloat16(nw);
}

__global__ void k_to_bf16(int64_t n, const float *w, __nv_bfloat16 *wb)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) wb[e] = __float2bfloat16(w[e]);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// per-column mean and standard deviation (FP64 sums; a floor keeps constant columns finite)
__global__ void k_colstats(int64_t M, int N, const float *X, float *mean, float *scale)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t m = 0; m < M; ++m) {
        const double v = X[m * N + n];
        s += v;
        s2 += v * v;
    }
    const double mu = s / (double)M;
    const double var = fmax(s2 / (double)M - mu * mu, 0.0);
    mean[n] = (float)mu;
    scale[n] = (float)fmax(sqrt(var), 1e-6);
}

__global__ void k_norm_out(int64_t n, const float *t, const float *mean, const float *scale,
                           float *y)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int f = (int)(e % NOUT);
    y[e] = (t[e] - mean[f]) / scale[f];
}

}  // namespace

// ---------------------------------------------------------------- host side

struct cq_guess {
    cq_ctx *ctx = nullptr;
    int n_layers = 4;                 // 3 hidden + output
    int dims[5] = {NDESC, 256, 256, 256, NOUT};
    bool fp32_weights = false;        // test mode: forward reads the FP32 weights
    DevBuf w, wb, b, gw, gb, mw, vw, mb, vb;  // all layers packed
    std::vector<int64_t> w_off, b_off;
    int64_t n_w = 0, n_b = 0;
    int64_t step = 0;
    DevBuf mean, scale;               // target normalisation (81 each)
    DevBuf in_mean, in_scale;         // descriptor normalisation (64 each)
    DevBuf xin;                       // normalised inputs of the current batch
    int64_t xin_rows = 0;
    DevBuf act;                       // Z and H per layer for a batch
    int64_t act_rows = 0;
    // tensor-core path (BF16 weights): W^T per layer (BF16, N x K), and BF16 copies of the
    // layer inputs, of dZ and the transposes H^T, dZ^T of the backward pass
    DevBuf wt, actb;
    int64_t actb_rows = 0;
    DevBuf loss_acc;                  // running squared-error sum and row count (2 doubles)
};

namespace {

cq_status ensure_act(cq_guess *g, int64_t rows)
{
    if (g->act_rows >= rows) return CQ_OK;
    int64_t per = 0;
    for (int l = 1; l <= g->n_layers; ++l) per += 2 * g->dims[l];
    per += g->dims[g->n_layers];  // dY
    per += 256;                   // dH scratch of the widest layer
    per += 256;
    CQ_TRY(cq_alloc(g->ctx, g->act, sizeof(float) * per * rows));
    g->act_rows = rows;
    return CQ_OK;
}

int64_t pad16(int64_t x) { return (x + 15) & ~(int64_t)15; }

// BF16 buffers of the tensor-core path for `rows` samples: layer inputs Hb[0..L-1]
// (rows x dims[l]), dZb (rows x 256), H^T and dZ^T (256 x pad16(rows) each)
cq_status ensure_actb(cq_guess *g, int64_t rows)
{
    if (g->actb_rows >= rows) return CQ_OK;
    int64_t per = 0;
    for (int l = 0; l < g->n_layers; ++l) per += g->dims[l];
    per += 256;
    const int64_t elems = per * rows + 2 * 256 * pad16(rows);
    CQ_TRY(cq_alloc(g->ctx, g->actb, sizeof(__nv_bfloat16) * elems));
    g->actb_rows = rows;
    return CQ_OK;
}

// W^T per layer in BF16 from the FP32 master weights (after every change of the weights)
void refresh_wt(cq_guess *g, cudaStream_t s)
{
    for (int l = 0; l < g->n_layers; ++l) {
        const int K = g->dims[l], N = g->dims[l + 1];
        k_to_bf16_mat<<<blocks_for((int64_t)K * N), 256, 0, s>>>(
            K, N, g->w.as<float>() + g->w_off[l], g->wt.as<__nv_bfloat16>() + g->w_off[l], 1, K);
    }
    cq_count_launch(g->n_layers);
}

cq_status tc_attr(cq_ctx *ctx)
{
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cq_fail(ctx, CQ_ERR_INVALID, "guess: device index");
    if (!done[dev]) {
        CQ_TRY(cq_check_cuda(ctx, cudaFuncSetAttribute(k_gemm_tc,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       TC_SMEM), "mlp attribute"));
        done[dev] = true;
    }
    return CQ_OK;
}

// C = A Bt^T on the tensor cores (see mlp_tc.cuh); parts > 1 splits K into that many
// deterministic partial products c_stride_z apart
void gemm_tc(cq_ctx *ctx, int M, int N, const __nv_bfloat16 *A, int64_t lda,
             const __nv_bfloat16 *Bt, int64_t ldb, float *C, int64_t ldc, int64_t K, int parts,
             int64_t c_stride_z)
{
    const int64_t chunk = parts > 1 ? pad16((K + parts - 1) / parts) : K;
    dim3 grid((unsigned)((M + TC_MT - 1) / TC_MT), (unsigned)((N + TC_NT - 1) / TC_NT),
              (unsigned)parts);
    k_gemm_tc<<<grid, 128, TC_SMEM, ctx->stream>>>(M, N, A, lda, Bt, ldb, C, ldc, 0, K,
                                                   c_stride_z, chunk, ctx->flag.as<int32_t>());
    cq_count_launch();
}

__global__ void k_norm_in(int64_t n, const float *x, const float *mean, const float *scale,
                          float *y)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int f = (int)(e % NDESC);
    y[e] = (x[e] - mean[f]) / scale[f];
}

// forward on `rows` descriptors (normalised first): H[n_layers] is the output (rows x 81)
cq_status mlp_forward(cq_guess *g, const float *X, int64_t rows, std::vector<float *> &Z,
                      std::vector<float *> &H)
{
    cq_ctx *ctx = g->ctx;
    CQ_TRY(ensure_act(g, rows));
    if (g->xin_rows < rows) {
        CQ_TRY(cq_alloc(ctx, g->xin, sizeof(float) * NDESC * rows));
        g->xin_rows = rows;
    }
    k_norm_in<<<blocks_for(rows * NDESC), 256, 0, ctx->stream>>>(
        rows * NDESC, X, g->in_mean.as<float>(), g->in_scale.as<float>(), g->xin.as<float>());
    cq_count_launch();
    float *base = g->act.as<float>();
    Z.assign(g->n_layers + 1, nullptr);
    H.assign(g->n_layers + 1, nullptr);
    H[0] = g->xin.as<float>();
    const bool tc = !g->fp32_weights;
    std::vector<__nv_bfloat16 *> Hb(g->n_layers, nullptr);
    if (tc) {
        // BF16 weights: the layers run on the tensor cores with BF16 inputs
        CQ_TRY(ensure_actb(g, rows));
        CQ_TRY(tc_attr(ctx));
        int64_t ob = 0;
        for (int l = 0; l < g->n_layers; ++l) {
            Hb[l] = g->actb.as<__nv_bfloat16>() + ob;
            ob += rows * g->dims[l];
        }
        k_to_bf16_mat<<<blocks_for(rows * NDESC), 256, 0, ctx->stream>>>(rows, NDESC, H[0],
                                                                          Hb[0], 0, 0);
        cq_count_launch();
    }
    int64_t off = 0;
    for (int l = 1; l <= g->n_layers; ++l) {
        Z[l] = base + off;
        off += rows * g->dims[l];
        H[l] = base + off;
        off += rows * g->dims[l];
        const int K = g->dims[l - 1], N = g->dims[l];
        if (tc) {
            gemm_tc(ctx, (int)rows, N, Hb[l - 1], K, g->wt.as<__nv_bfloat16>() + g->w_off[l - 1], K,
                    Z[l], N, K, 1, 0);
        } else {
            dim3 grid((N + 63) / 64, (unsigned)((rows + 63) / 64), 1);
            k_gemm<false, false, float><<<grid, 256, 0, ctx->stream>>>(
                (int)rows, N, H[l - 1], K, g->w.as<float>() + g->w_off[l - 1], N, Z[l], N, 0, K, 0,
                K);
            cq_count_launch();
        }
        k_bias_act<<<blocks_for(rows * N), 256, 0, ctx->stream>>>(
            rows, N, g->b.as<float>() + g->b_off[l - 1], Z[l], H[l], l < g->n_layers ? 1 : 0,
            tc && l < g->n_layers ? Hb[l] : nullptr);
        cq_count_launch();
    }
    return cq_check_cuda(ctx, cudaGetLastError(), "mlp forward");
}

}  // namespace

extern "C" cq_status cq_guess_create(cq_ctx *ctx, uint64_t seed, int32_t fp32_weights,
                                     cq_guess **out)
{
    if (!ctx || !out) return CQ_ERR_INVALID;
    std::unique_ptr<cq_guess> g(new cq_guess());
    g->ctx = ctx;
    g->fp32_weights = fp32_weights != 0;
    g->w_off.push_back(0);
    g->b_off.push_back(0);
    for (int l = 0; l < g->n_layers; ++l) {
        g->w_off.push_back(g->w_off.back() + (int64_t)g->dims[l] * g->dims[l + 1]);
        g->b_off.push_back(g->b_off.back() + g->dims[l + 1]);
    }
    g->n_w = g->w_off.back();
    g->n_b = g->b_off.back();
    for (DevBuf *b : {&g->w, &g->gw, &g->mw, &g->vw})
        CQ_TRY(cq_alloc(ctx, *b, sizeof(float) * g->n_w));
    for (DevBuf *b : {&g->b, &g->gb, &g->mb, &g->vb})
        CQ_TRY(cq_alloc(ctx, *b, sizeof(float) * g->n_b));
    CQ_TRY(cq_alloc(ctx, g->wb, sizeof(__nv_bfloat16) * g->n_w));
    CQ_TRY(cq_alloc(ctx, g->wt, sizeof(__nv_bfloat16) * g->n_w));
    CQ_TRY(cq_alloc(ctx, g->mean, sizeof(float) * NOUT));
    CQ_TRY(cq_alloc(ctx, g->scale, sizeof(float) * NOUT));
    CQ_TRY(cq_alloc(ctx, g->in_mean, sizeof(float) * NDESC));
    CQ_TRY(cq_alloc(ctx, g->in_scale, sizeof(float) * NDESC));
    // He-style initialisation from a seeded generator (host), zero biases and moments
    std::mt19937_64 rng(seed);
    std::vector<float> w(g->n_w);
    for (int l = 0; l < g->n_layers; ++l) {
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / g->dims[l]) *
                                                    (l + 1 == g->n_layers ? 0.1f : 1.f));
        for (int64_t e = g->w_off[l]; e < g->w_off[l + 1]; ++e) w[e] = nd(rng);
    }
    cudaStream_t s = ctx->stream;
    cudaMemcpyAsync(g->w.ptr, w.data(), sizeof(float) * g->n_w, cudaMemcpyHostToDevice, s);
    for (DevBuf *b : {&g->mw, &g->vw}) cudaMemsetAsync(b->ptr, 0, sizeof(float) * g->n_w, s);
    for (DevBuf *b : {&g->b, &g->mb, &g->vb}) cudaMemsetAsync(b->ptr, 0, sizeof(float) * g->n_b, s);
    std::vector<float> zero(NOUT, 0.f), one(NOUT, 1.f);
    cudaMemcpyAsync(g->mean.ptr, zero.data(), sizeof(float) * NOUT, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->scale.ptr, one.data(), sizeof(float) * NOUT, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->in_mean.ptr, zero.data(), sizeof(float) * NDESC, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->in_scale.ptr, one.data(), sizeof(float) * NDESC, cudaMemcpyHostToDevice, s);
    k_to_bf16<<<blocks_for(g->n_w), 256, 0, s>>>(g->n_w, g->w.as<float>(), g->wb.as<__nv_bfloat16>());
    cq_count_launch();
    refresh_wt(g.get(), s);
    CQ_TRY(cq_check_cuda(ctx, cudaStreamSynchronize(s), "guess create"));
    *out = g.release();
    return CQ_OK;
}

extern "C" void cq_guess_destroy(cq_guess *g)
{
    if (!g) return;
    if (g->ctx) cudaStreamSynchronize(g->ctx->stream);
    delete g;
}

extern "C" cq_status cq_guess_params(cq_guess *g, float *w_host, float *b_host, int64_t *n_w,
                                     int64_t *n_b, int32_t set)
{
    if (!g) return CQ_ERR_INVALID;
    if (n_w) *n_w = g->n_w;
    if (n_b) *n_b = g->n_b;
    cudaStream_t s = g->ctx->stream;
    if (set) {
        if (w_host) cudaMemcpyAsync(g->w.ptr, w_host, 4 * g->n_w, cudaMemcpyHostToDevice, s);
        if (b_host) cudaMemcpyAsync(g->b.ptr, b_host, 4 * g->n_b, cudaMemcpyHostToDevice, s);
        k_to_bf16<<<blocks_for(g->n_w), 256, 0, s>>>(g->n_w, g->w.as<float>(),
                                                      g->wb.as<__nv_bfloat16>());
        cq_count_launch();
        refresh_wt(g, s);
    } else {
        if (w_host) cudaMemcpyAsync(w_host, g->w.ptr, 4 * g->n_w, cudaMemcpyDeviceToHost, s);
        if (b_host) cudaMemcpyAsync(b_host, g->b.ptr, 4 * g->n_b, cudaMemcpyDeviceToHost, s);
    }
    return cq_check_cuda(g->ctx, cudaStreamSynchronize(s), "guess params");
}

extern "C" cq_status cq_guess_fit_scale(cq_guess *g, const float *desc, const float *targets,
                                        int64_t rows)
{
    if (!g || !desc || !targets || rows <= 0) return CQ_ERR_INVALID;
    cudaStream_t s = g->ctx->stream;
    k_colstats<<<1, 128, 0, s>>>(rows, NDESC, desc, g->in_mean.as<float>(), g->in_scale.as<float>());
    k_colstats<<<1, 128, 0, s>>>(rows, NOUT, targets, g->mean.as<float>(), g->scale.as<float>());
    cq_count_launch(2);
    return cq_check_cuda(g->ctx, cudaStreamSynchronize(s), "fit scale");
}

extern "C" cq_status cq_guess_set_scale(cq_guess *g, const float *in_mean_host,
                                        const float *in_scale_host, const float *out_mean_host,
                                        const float *out_scale_host)
{
    if (!g || !in_mean_host || !in_scale_host || !out_mean_host || !out_scale_host)
        return CQ_ERR_INVALID;
    cudaStream_t s = g->ctx->stream;
    cudaMemcpyAsync(g->in_mean.ptr, in_mean_host, 4 * NDESC, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->in_scale.ptr, in_scale_host, 4 * NDESC, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->mean.ptr, out_mean_host, 4 * NOUT, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(g->scale.ptr, out_scale_host, 4 * NOUT, cudaMemcpyHostToDevice, s);
    return cq_check_cuda(g->ctx, cudaStreamSynchronize(s), "guess scale");
}

static cq_status pair_list(cq_ctx *ctx, const cq_pattern *pL, int32_t **pairs, int64_t *n)
{
    const int64_t nblk = pL->n_blocks;
    void *vf, *vp, *vl;
    CQ_TRY(cq_scratch(ctx, "gs_flags", 8 * (nblk + 1), &vf));
    CQ_TRY(cq_scratch(ctx, "gs_pos", 8 * (nblk + 1), &vp));
    k_pair_flags<<<blocks_for(nblk), 256, 0, ctx->stream>>>(nblk, pL->row.as<int32_t>(),
                                                            pL->col.as<int32_t>(), (int64_t *)vf);
    cq_count_launch();
    CQ_TRY(cq_scan_i64(ctx, (int64_t *)vf, (int64_t *)vp, nblk));
    cudaMemcpyAsync(n, (int64_t *)vp + nblk, 8, cudaMemcpyDeviceToHost, ctx->stream);
    CQ_TRY(cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "pairs"));
    CQ_TRY(cq_scratch(ctx, "gs_pairs", 4 * (*n + 1), &vl));
    k_pair_fill<<<blocks_for(nblk), 256, 0, ctx->stream>>>(nblk, pL->row.as<int32_t>(),
                                                           pL->col.as<int32_t>(), (int64_t *)vp,
                                                           (int32_t *)vl);
    cq_count_launch();
    *pairs = (int32_t *)vl;
    return cq_check_cuda(ctx, cudaGetLastError(), "pairs");
}

extern "C" cq_status cq_guess_pairs(cq_ctx *ctx, const cq_pattern *pL, int64_t *n_pairs_host)
{
    if (!ctx || !pL || !n_pairs_host) return CQ_ERR_INVALID;
    int32_t *pairs;
    return pair_list(ctx, pL, &pairs, n_pairs_host);
}

extern "C" cq_status cq_guess_descriptors(cq_ctx *ctx, const cq_pattern *pL, float *desc,
                                          float *frames, int32_t *pairs_out)
{
    if (!ctx || !pL || !desc || !frames) return CQ_ERR_INVALID;
    if (pL->n_cells() != 1)
        return cq_fail(ctx, CQ_ERR_INVALID, "guess: single-cell patterns only");
    int32_t *pairs;
    int64_t n;
    CQ_TRY(pair_list(ctx, pL, &pairs, &n));
    if (n == 0) return CQ_OK;
    Box3 box;
    for (int c = 0; c < 3; ++c) box.v[c] = pL->geo->box[c];
    k_descriptors<<<blocks_for(n, 128), 128, 0, ctx->stream>>>(
        n, pairs, pL->row.as<int32_t>(), pL->col.as<int32_t>(), pL->row_ptr.as<int64_t>(),
        pL->geo->pos.as<double>(), box, desc, frames);
    cq_count_launch();
    if (pairs_out)
        cudaMemcpyAsync(pairs_out, pairs, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream);
    return cq_check_cuda(ctx, cudaGetLastError(), "descriptors");
}

extern "C" cq_status cq_guess_targets(cq_ctx *ctx, const cq_pattern *pL, const double *L,
                                      const float *frames, float *targets)
{
    if (!ctx || !pL || !L || !frames || !targets) return CQ_ERR_INVALID;
    const int nb = pL->geo->uniform_nb;
    if (nb != 9 && nb != 4) return cq_fail(ctx, CQ_ERR_INVALID, "guess: uniform 4 or 9 orbitals");
    int32_t *pairs;
    int64_t n;
    CQ_TRY(pair_list(ctx, pL, &pairs, &n));
    if (n == 0) return CQ_OK;
    k_targets<<<blocks_for(n, 128), 128, 0, ctx->stream>>>(n, nb, pL->uniform, pairs, frames, L,
                                                           targets);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "targets");
}

extern "C" cq_status cq_guess_forward(cq_guess *g, const float *desc, int64_t rows, float *out)
{
    if (!g || !desc || !out || rows < 0) return CQ_ERR_INVALID;
    if (rows == 0) return CQ_OK;
    std::vector<float *> Z, H;
    CQ_TRY(mlp_forward(g, desc, rows, Z, H));
    return cq_check_cuda(g->ctx, cudaMemcpyAsync(out, H[g->n_layers], 4 * rows * NOUT,
                                                 cudaMemcpyDeviceToDevice, g->ctx->stream),
                         "forward copy");
}

// One optimisation step on a minibatch: forward, MSE against normalised targets, backward
// (deterministic: the weight-gradient reduction over rows is split into fixed chunks and
// summed in order), Adam.  lr = 0 computes the loss and gradients without an update.
extern "C" cq_status cq_guess_train_step(cq_guess *g, const float *desc, const float *targets,
                                         int64_t rows, float lr, float *loss_host,
                                         float *grad_w_host, float *grad_b_host)
{
    if (!g || !desc || !targets || rows <= 0) return CQ_ERR_INVALID;
    cq_ctx *ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    std::vector<float *> Z, H;
    CQ_TRY(mlp_forward(g, desc, rows, Z, H));
    const int L = g->n_layers;
    void *vdy, *vdh, *vpart, *vloss;
    int64_t maxw = 0;
    for (int l = 0; l <= L; ++l) maxw = std::max<int64_t>(maxw, g->dims[l]);
    CQ_TRY(cq_scratch(ctx, "gs_dy", 4 * rows * maxw, &vdy));
    CQ_TRY(cq_scratch(ctx, "gs_dh", 4 * rows * maxw, &vdh));
    const int parts = 16;
    CQ_TRY(cq_scratch(ctx, "gs_part", 4 * (int64_t)parts * 256 * 256, &vpart));
    CQ_TRY(cq_scratch(ctx, "gs_loss", 4 * 256, &vloss));
    float *dY = (float *)vdy, *dH = (float *)vdh;
    void *vt;
    CQ_TRY(cq_scratch(ctx, "gs_tnorm", 4 * rows * NOUT, &vt));
    k_norm_out<<<blocks_for(rows * NOUT), 256, 0, s>>>(rows * NOUT, targets, g->mean.as<float>(),
                                                      g->scale.as<float>(), (float *)vt);
    k_mse<<<256, 256, 0, s>>>(rows, H[L], (float *)vt, dY, (float *)vloss);
    if (!g->loss_acc.ptr) {
        CQ_TRY(cq_alloc(ctx, g->loss_acc, 2 * sizeof(double)));
        CQ_TRY(cq_check_cuda(ctx, cudaMemsetAsync(g->loss_acc.ptr, 0, 2 * sizeof(double), s),
                             "loss sums"));
    }
    k_loss_accum<<<1, 256, 0, s>>>((const float *)vloss, rows, g->loss_acc.as<double>());
    cq_count_launch(3);
    // dY holds dLoss/dZ_L (output layer is linear)
    float *dZ = dY;
    const bool tc = !g->fp32_weights;
    __nv_bfloat16 *dZb = nullptr, *Ht = nullptr, *dZt = nullptr;
    const int64_t rp = pad16(rows);
    if (tc) {
        int64_t ob = 0;
        for (int l = 0; l < L; ++l) ob += rows * g->dims[l];
        dZb = g->actb.as<__nv_bfloat16>() + ob;
        Ht = dZb + rows * 256;
        dZt = Ht + 256 * rp;
    }
    for (int l = L; l >= 1; --l) {
        const int K = g->dims[l - 1], N = g->dims[l];
        // dW_l = H_{l-1}^T dZ  (K x N), reduction over rows in `parts` fixed chunks
        const int64_t chunk = ((rows + parts - 1) / parts + 15) / 16 * 16;
        if (tc) {
            // tensor cores: dW = (H^T)(dZ^T)^T from BF16 transposes (rows padded to 16)
            const dim3 tb(32, 8);
            k_to_bf16_t<<<dim3((K + 31) / 32, (unsigned)((rows + 31) / 32)), tb, 0, s>>>(
                rows, K, H[l - 1], Ht, rp);
            k_to_bf16_t<<<dim3((N + 31) / 32, (unsigned)((rows + 31) / 32)), tb, 0, s>>>(
                rows, N, dZ, dZt, rp);
            cq_count_launch(2);
            gemm_tc(ctx, K, N, Ht, rp, dZt, rp, (float *)vpart, N, rows, parts, (int64_t)K * N);
        } else {
            dim3 grid((N + 63) / 64, (K + 63) / 64, parts);
            k_gemm<true, false, float><<<grid, 256, 0, s>>>(K, N, H[l - 1], K, dZ, N,
                                                            (float *)vpart, N, 0, rows,
                                                            (int64_t)K * N, chunk);
            cq_count_launch();
        }
        k_sum_parts<<<blocks_for((int64_t)K * N), 256, 0, s>>>((int64_t)K * N, parts,
                                                             (int64_t)K * N, (float *)vpart,
                                                             g->gw.as<float>() + g->w_off[l - 1]);
        k_colsum<<<blocks_for(N), 256, 0, s>>>(rows, N, dZ, g->gb.as<float>() + g->b_off[l - 1]);
        cq_count_launch(2);
        if (l > 1) {
            // dH_{l-1} = dZ W_l^T (rows x K), then dZ_{l-1} = dH * silu'(Z_{l-1})
            if (tc) {
                // W (K x N, row-major) is already the K-major second operand of dZ W^T
                k_to_bf16_mat<<<blocks_for(rows * N), 256, 0, s>>>(rows, N, dZ, dZb, 0, 0);
                cq_count_launch();
                gemm_tc(ctx, (int)rows, K, dZb, N, g->wb.as<__nv_bfloat16>() + g->w_off[l - 1], N,
                        dH, K, N, 1, 0);
            } else {
                dim3 g2((K + 63) / 64, (unsigned)((rows + 63) / 64), 1);
                k_gemm<false, true, float><<<g2, 256, 0, s>>>(
                    (int)rows, K, dZ, N, g->w.as<float>() + g->w_off[l - 1], N, dH, K, 0, N, 0, N);
                cq_count_launch();
            }
            // dZ of layer l is no longer needed: the next layer's dZ reuses its buffer
            k_act_back<<<blocks_for(rows * K), 256, 0, s>>>(rows * K, Z[l - 1], dH, dY);
            cq_count_launch();
            dZ = dY;
        }
    }
    CQ_TRY(cq_check_cuda(ctx, cudaGetLastError(), "mlp backward"));
    if (lr > 0.f) {
        g->step += 1;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - std::pow(b1, (float)g->step), c2 = 1.f - std::pow(b2, (float)g->step);
        k_adam<<<blocks_for(g->n_w), 256, 0, s>>>(g->n_w, g->w.as<float>(), g->gw.as<float>(),
                                                  g->mw.as<float>(), g->vw.as<float>(),
                                                  g->wb.as<__nv_bfloat16>(), lr, b1, b2, eps, c1, c2);
        k_adam<<<blocks_for(g->n_b), 256, 0, s>>>(g->n_b, g->b.as<float>(), g->gb.as<float>(),
                                                  g->mb.as<float>(), g->vb.as<float>(), nullptr, lr,
                                                  b1, b2, eps, c1, c2);
        cq_count_launch(2);
        refresh_wt(g, s);
    }
    if (loss_host) {
        float part[256];
        cudaMemcpyAsync(part, vloss, sizeof(part), cudaMemcpyDeviceToHost, s);
        CQ_TRY(cq_check_cuda(ctx, cudaStreamSynchronize(s), "loss"));
        double tot = 0.0;
        for (int q = 0; q < 256; ++q) tot += part[q];
        *loss_host = (float)(tot / ((double)rows * NOUT));
    }
    if (grad_w_host)
        cudaMemcpyAsync(grad_w_host, g->gw.ptr, 4 * g->n_w, cudaMemcpyDeviceToHost, s);
    if (grad_b_host)
        cudaMemcpyAsync(grad_b_host, g->gb.ptr, 4 * g->n_b, cudaMemcpyDeviceToHost, s);
    if (!loss_host && !grad_w_host && !grad_b_host)
        return cq_check_cuda(ctx, cudaGetLastError(), "train step");
    return cq_check_cuda(ctx, cudaStreamSynchronize(s), "train step");
}

extern "C" cq_status cq_guess_loss_sum(cq_guess *g, double *sq_sum_host, int64_t *rows_host,
                                       int32_t reset)
{
    if (!g) return CQ_ERR_INVALID;
    cq_ctx *ctx = g->ctx;
    double v[2] = {0.0, 0.0};
    if (g->loss_acc.ptr) {
        cudaMemcpyAsync(v, g->loss_acc.ptr, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream);
        if (reset) cudaMemsetAsync(g->loss_acc.ptr, 0, sizeof(v), ctx->stream);
        CQ_TRY(cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "loss sums"));
    }
    if (sq_sum_host) *sq_sum_host = v[0];
    if (rows_host) *rows_host = (int64_t)v[1];
    return CQ_OK;
}

// Predict every block of P_L: descriptors -> MLP -> un-normalise -> rotate to the global
// frame; writes all (i, j) and (j, i) blocks of L.
extern "C" cq_status cq_guess_apply(cq_guess *g, const cq_pattern *pL, double *L)
{
    if (!g || !pL || !L) return CQ_ERR_INVALID;
    cq_ctx *ctx = g->ctx;
    const int nb = pL->geo->uniform_nb;
    if (nb != 9 && nb != 4) return cq_fail(ctx, CQ_ERR_INVALID, "guess: uniform 4 or 9 orbitals");
    int64_t n;
    int32_t *pairs;
    CQ_TRY(pair_list(ctx, pL, &pairs, &n));
    void *vd, *vf, *vo, *vp;
    CQ_TRY(cq_scratch(ctx, "ga_desc", 4 * (n + 1) * NDESC, &vd));
    CQ_TRY(cq_scratch(ctx, "ga_frames", 4 * (n + 1) * 9, &vf));
    CQ_TRY(cq_scratch(ctx, "ga_out", 4 * (n + 1) * NOUT, &vo));
    CQ_TRY(cq_scratch(ctx, "ga_pairs", 4 * (n + 1), &vp));
    CQ_TRY(cq_guess_descriptors(ctx, pL, (float *)vd, (float *)vf, (int32_t *)vp));
    // forward in row chunks that keep the activations modest
    const int64_t chunk = 1 << 18;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        CQ_TRY(cq_guess_forward(g, (float *)vd + r0 * NDESC, rows, (float *)vo + r0 * NOUT));
    }
    CQ_TRY(cq_check_cuda(ctx, cudaMemsetAsync(L, 0, sizeof(double) * pL->n_values, ctx->stream),
                         "apply"));
    k_apply<<<blocks_for(n, 128), 128, 0, ctx->stream>>>(
        n, nb, pL->uniform, (int32_t *)vp, pL->transpose.as<int64_t>(), (float *)vf, (float *)vo,
        g->mean.as<float>(), g->scale.as<float>(), L);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "apply");
}
