// Split-BF16 block-sparse product on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// C <- beta C + alpha mask_{P_C}(A.B) with every FP64 operand value split into three BF16
// terms x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); the
// residuals are exact in FP64) and the product formed as the six cross products
// A_p B_q with p + q <= 2, accumulated in FP32 in tensor memory.  Every DRAIN chunks the
// FP32 accumulator is drained into a per-thread double-float (hi, lo) sum, so FP32
// rounding only acts within a drain period; the result is written back in FP64.
//
// Local densification.  9x9 blocks do not fit MMA shapes, so atoms are grouped in space
// (Morton order): an M tile is a group of floor(128/nb) atoms (126 rows for nb = 9), an N
// tile a group of floor(64/nb) atoms.  A work tile is a pair (M group g, N group h) that
// holds at least one block of P_C; its K list is every atom k with (i, k) in P_A for some
// i in g and (k, j) in P_B for some j in h (built on the device with shared-memory
// bitmaps).  Absent blocks are zero in shared memory.  Every C block belongs to exactly one
// tile, so there are no atomics.
//
// K layout.  Along K an atom's orbitals are split into a "main" piece of 8 values (one
// 16-byte core-matrix row) and a "tail" of 4 values (half a core-matrix row; for nb = 9:
// orbital 8 and three zeros, for nb = 4: all four orbitals).  A K chunk of 48 values (six
// core-matrix columns, three MMA K steps) holds 4 atoms of 9 orbitals (mains in columns
// 0-3, tails paired in columns 4-5) or 12 atoms of 4 orbitals (tails only), so 9-orbital
// atoms cost 12 K values instead of 16.
//
// Operands are pre-split once per product into BF16 planes ("A form": rows = left orbital,
// K = right orbital; "B form": rows = right orbital, K = left orbital), each as a main
// array (8 values per block row) and a tail array (4 values per block row), so the tile
// kernel only moves aligned 16- and 8-byte pieces with cp.async into the canonical
// no-swizzle K-major layout (core matrix = 8 rows x 16 bytes; LBO = 128 B between
// K-adjacent core matrices, SBO = 768 B between 8-row groups) and one thread issues the
// MMAs.  Producer warps, the MMA thread and the drain warps hand stages and the two TMEM
// accumulators to one another through mbarriers (bsmm_split_kernel.cuh).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "cq_internal.cuh"

namespace {

constexpr int ST = 384;                      // threads per CTA (12 warps)
constexpr int MT = 128, NT = 64, KCH = 48;   // tile M, N and K chunk
constexpr int KSTEPS = KCH / 16;             // MMA K steps per chunk
constexpr int TAILW = 4;                     // values in an atom's tail piece
constexpr int SBO = (KCH / 8) * 128;         // bytes between 8-row groups
constexpr int A_PLANE = MT * KCH * 2;        // 12 KB
constexpr int B_PLANE = NT * KCH * 2;        // 6 KB
constexpr int STAGE = 3 * A_PLANE + 3 * B_PLANE;
constexpr int BAR_BYTES = 256;
constexpr int DRAIN = 4;                     // chunks per FP32 accumulation period
constexpr int TMEM_COLS = 2 * NT;            // two FP32 accumulators
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// Atoms per chunk and core-matrix columns of an atom's pieces.
template <int NB> struct KLayout;
template <> struct KLayout<9> {
    static constexpr int CA = 4, MAINW = 8;
    __device__ static constexpr int main_col(int a) { return a; }
    __device__ static constexpr int tail_col(int a) { return 4 + (a >> 1); }
};
template <> struct KLayout<4> {
    static constexpr int CA = 12, MAINW = 0;
    __device__ static constexpr int main_col(int) { return 0; }
    __device__ static constexpr int tail_col(int a) { return a >> 1; }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (row, core-matrix column, byte) in the canonical no-swizzle K-major layout
__device__ __forceinline__ uint32_t tile_off(int row, int col, int byte)
{
    return (uint32_t)((row >> 3) * SBO + col * 128 + (row & 7) * 16 + byte);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;    // leading (K) byte offset
    d |= (uint64_t)(SBO >> 4) << 32;    // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    return d;                           // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(MT >> 4) << 24);

__device__ __forceinline__ void split3(double x, __nv_bfloat16 &b0, __nv_bfloat16 &b1,
                                       __nv_bfloat16 &b2)
{
    b0 = __double2bfloat16(x);
    double r = x - (double)__bfloat162float(b0);
    b1 = __double2bfloat16(r);
    r = r - (double)__bfloat162float(b1);
    b2 = __double2bfloat16(r);
}

struct SplitPlanes {
    __nv_bfloat16 *main[3], *tail[3];
};

// Position of K value m of a block row in the main/tail arrays of a plane.
__device__ __forceinline__ int64_t piece_index(int64_t row, int m, int mainw, int64_t n_rows,
                                               bool &in_tail)
{
    in_tail = m >= mainw;
    return in_tail ? row * TAILW + (m - mainw) : row * mainw + m;
}

// A form: block b = (i, k) -> row r < nb (orbital of i), K value m (orbital of k).
// One thread per (block, row, m < mainw + 4); writes three planes of main and tail arrays.
__global__ void k_split_a(int64_t n, int nb, int mainw, int stride, const double *__restrict__ A,
                          SplitPlanes out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int ka = mainw + TAILW;
    const int64_t row = e / ka;
    const int m = (int)(e - row * ka);
    const int64_t b = row / nb;
    const int r = (int)(row - b * nb);
    const double x = m < nb ? A[b * stride + r * nb + m] : 0.0;
    bool in_tail;
    const int64_t q = piece_index(row, m, mainw, 0, in_tail);
    __nv_bfloat16 v[3];
    split3(x, v[0], v[1], v[2]);
    for (int pl = 0; pl < 3; ++pl) (in_tail ? out.tail[pl] : out.main[pl])[q] = v[pl];
}

// B form: block b = (k, j) -> row n < nb (orbital of j), K value m (orbital of k).
__global__ void k_split_b(int64_t n, int nb, int mainw, int stride, const double *__restrict__ B,
                          SplitPlanes out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int ka = mainw + TAILW;
    const int64_t row = e / ka;
    const int m = (int)(e - row * ka);
    const int64_t b = row / nb;
    const int r = (int)(row - b * nb);
    const double x = m < nb ? B[b * stride + m * nb + r] : 0.0;
    bool in_tail;
    const int64_t q = piece_index(row, m, mainw, 0, in_tail);
    __nv_bfloat16 v[3];
    split3(x, v[0], v[1], v[2]);
    for (int pl = 0; pl < 3; ++pl) (in_tail ? out.tail[pl] : out.main[pl])[q] = v[pl];
}

// Tile existence: bit (g, h) for every C block (i, j).
__global__ void k_tile_mark(int64_t n_c, const int32_t *c_row, const int32_t *c_col,
                            const int32_t *g_of, const int32_t *h_of, int n_h, uint32_t *bits)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_c) return;
    const int64_t key = (int64_t)g_of[c_row[b]] * n_h + h_of[c_col[b]];
    atomicOr(&bits[key >> 5], 1u << (key & 31));
}

// K list of each tile: atoms k reachable from the M group through P_A and from the N group
// through P_B (P_B symmetric: (k, j) in P_B <=> k in row j).  COUNT pass writes sizes,
// the FILL pass writes ascending atom indices.
template <bool FILL>
__global__ void __launch_bounds__(256)
k_tile_klist(int n_atoms, const int2 *tiles, int gi, int gj, const int32_t *g_atoms,
             const int32_t *h_atoms, const int64_t *a_rp, const int32_t *a_col,
             const int64_t *b_rp, const int32_t *b_col, int64_t *count, const int64_t *start,
             int32_t *klist)
{
    extern __shared__ uint32_t bm[];  // 2 * words
    const int words = (n_atoms + 31) >> 5;
    uint32_t *ba = bm, *bb = bm + words;
    for (int w = threadIdx.x; w < 2 * words; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int2 t = tiles[blockIdx.x];
    for (int s = 0; s < gi; ++s) {
        const int i = g_atoms[(int64_t)t.x * gi + s];
        if (i < 0) continue;
        for (int64_t e = a_rp[i] + threadIdx.x; e < a_rp[i + 1]; e += blockDim.x) {
            const int k = a_col[e];
            atomicOr(&ba[k >> 5], 1u << (k & 31));
        }
    }
    for (int s = 0; s < gj; ++s) {
        const int j = h_atoms[(int64_t)t.y * gj + s];
        if (j < 0) continue;
        for (int64_t e = b_rp[j] + threadIdx.x; e < b_rp[j + 1]; e += blockDim.x) {
            const int k = b_col[e];
            atomicOr(&bb[k >> 5], 1u << (k & 31));
        }
    }
    __syncthreads();
    // each thread owns a contiguous run of words
    const int per = (words + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
    int mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(ba[w] & bb[w]);
    __shared__ int scan[256];
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (!FILL) {
        if (threadIdx.x == blockDim.x - 1) count[blockIdx.x] = scan[threadIdx.x];
        return;
    }
    int64_t out = start[blockIdx.x] + scan[threadIdx.x] - mine;
    for (int w = w0; w < w1; ++w) {
        uint32_t v = ba[w] & bb[w];
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            klist[out++] = w * 32 + bit;
        }
    }
}

// Block-index table of each tile: for every K-list entry k and every slot s of the tile's
// groups, the index of block (i_s, k) in P_A (s < gi) or of block (k, j_s) in P_B, else -1.
// Built once per pattern triple so the product kernel's gather has no dependent searches.
__global__ void __launch_bounds__(256)
k_tile_index(const int2 *tiles, int gi, int gj, const int32_t *g_atoms, const int32_t *h_atoms,
             const int64_t *a_rp, const int32_t *a_col, const int64_t *b_rp,
             const int32_t *b_col, const int64_t *b_tr, const int64_t *kstart,
             const int32_t *klist, int32_t *table)
{
    const int2 t = tiles[blockIdx.x];
    const int64_t kb = kstart[blockIdx.x], kn = kstart[blockIdx.x + 1] - kb;
    const int w = gi + gj;
    for (int s = 0; s < w; ++s) {
        const bool left = s < gi;
        const int atom = left ? g_atoms[(int64_t)t.x * gi + s] : h_atoms[(int64_t)t.y * gj + s - gi];
        const int64_t *rp = left ? a_rp : b_rp;
        const int32_t *cl = left ? a_col : b_col;
        for (int64_t q = threadIdx.x; q < kn; q += blockDim.x) {
            int32_t idx = -1;
            if (atom >= 0) {
                const int k = klist[kb + q];
                int64_t lo = rp[atom], hi = rp[atom + 1];
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (cl[mid] < k)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (lo < rp[atom + 1] && cl[lo] == k) idx = (int32_t)(left ? lo : b_tr[lo]);
            }
            table[(kb + q) * w + s] = idx;
        }
    }
}

// cp.async of 16 or 8 bytes; src_bytes = 0 writes zeros and reads nothing
__device__ __forceinline__ void cp16z(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp8z(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

struct SplitArgs {
    int n_tiles;
    const int2 *tiles;
    const int64_t *kstart;
    const int32_t *klist;
    const int32_t *table;
    const int32_t *g_atoms, *h_atoms;
    const int64_t *a_rp, *b_rp, *c_rp;
    const int32_t *a_col, *b_col, *c_col;
    const int64_t *b_tr;
    const __nv_bfloat16 *sa_main[3], *sa_tail[3], *sb_main[3], *sb_tail[3];
    double *C;
    int c_stride;
    double alpha, beta;
    int32_t *flag;
};

#include "bsmm_split_kernel.cuh"

constexpr int SMEM = NS * STAGE + BAR_BYTES;  // pipeline stages + barriers

// ---------------------------------------------------------------- host side

struct Groups {
    int gi = 0, gj = 0, n_g = 0, n_h = 0, ca = 0;  // atoms per M, N group; atoms per K chunk
    DevBuf g_atoms, h_atoms, g_of, h_of;
};

struct SplitTiles {
    int n_tiles = 0;
    int64_t n_k = 0;
    double mma_flops = 0.0;  // tensor-core flops of one product over these tiles
    DevBuf tiles, kstart, klist, table;
};

// Morton order of the atoms (positions quantised to 1024 per box edge).
std::vector<int32_t> spatial_order(const Geometry &g)
{
    auto spread = [](uint64_t v) {
        uint64_t x = v & 0x3ff;
        x = (x | (x << 16)) & 0x30000ff;
        x = (x | (x << 8)) & 0x300f00f;
        x = (x | (x << 4)) & 0x30c30c3;
        x = (x | (x << 2)) & 0x9249249;
        return x;
    };
    std::vector<uint64_t> key(g.n_atoms);
    for (int i = 0; i < g.n_atoms; ++i) {
        uint64_t c[3];
        for (int d = 0; d < 3; ++d) {
            double f = g.pos_host[3 * i + d] / g.box[d];
            f -= std::floor(f);
            c[d] = (uint64_t)std::min(1023.0, std::max(0.0, f * 1024.0));
        }
        key[i] = spread(c[0]) | (spread(c[1]) << 1) | (spread(c[2]) << 2);
    }
    std::vector<int32_t> order(g.n_atoms);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return key[x] < key[y]; });
    return order;
}

cq_status get_groups(cq_ctx *ctx, const cq_pattern *p, Groups **out)
{
    auto key = std::make_tuple(1, p->geo->id, (uint64_t)0, (uint64_t)0);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<Groups *>(it->second.get());
        return CQ_OK;
    }
    const Geometry &g = *p->geo;
    auto gr = std::make_shared<Groups>();
    const int nb = g.uniform_nb;
    gr->gi = MT / nb;
    gr->gj = NT / nb;
    gr->ca = nb == 9 ? KLayout<9>::CA : KLayout<4>::CA;
    gr->n_g = (g.n_atoms + gr->gi - 1) / gr->gi;
    gr->n_h = (g.n_atoms + gr->gj - 1) / gr->gj;
    std::vector<int32_t> order = spatial_order(g);
    std::vector<int32_t> ga((size_t)gr->n_g * gr->gi, -1), ha((size_t)gr->n_h * gr->gj, -1);
    std::vector<int32_t> gof(g.n_atoms), hof(g.n_atoms);
    for (int r = 0; r < g.n_atoms; ++r) {
        ga[r] = order[r];
        gof[order[r]] = r / gr->gi;
        ha[r] = order[r];
        hof[order[r]] = r / gr->gj;
    }
    cq_status st;
    if ((st = cq_alloc(ctx, gr->g_atoms, 4 * ga.size())) != CQ_OK ||
        (st = cq_alloc(ctx, gr->h_atoms, 4 * ha.size())) != CQ_OK ||
        (st = cq_alloc(ctx, gr->g_of, 4 * gof.size())) != CQ_OK ||
        (st = cq_alloc(ctx, gr->h_of, 4 * hof.size())) != CQ_OK)
        return st;
    cudaMemcpyAsync(gr->g_atoms.ptr, ga.data(), 4 * ga.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(gr->h_atoms.ptr, ha.data(), 4 * ha.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(gr->g_of.ptr, gof.data(), 4 * gof.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(gr->h_of.ptr, hof.data(), 4 * hof.size(), cudaMemcpyHostToDevice, ctx->stream);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "groups")) != CQ_OK) return st;
    *out = gr.get();
    ctx->aux[key] = gr;
    return CQ_OK;
}

cq_status get_tiles(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                    const cq_pattern *pC, const Groups *gr, SplitTiles **out)
{
    auto key = std::make_tuple(2, pA->id, pB->id, pC->id);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<SplitTiles *>(it->second.get());
        return CQ_OK;
    }
    cudaStream_t s = ctx->stream;
    auto st_ = std::make_shared<SplitTiles>();
    const int64_t nbits = (int64_t)gr->n_g * gr->n_h;
    const int64_t nwords = (nbits + 31) / 32;
    void *vb;
    cq_status st = cq_scratch(ctx, "split_bits", 4 * nwords, &vb);
    if (st != CQ_OK) return st;
    cudaMemsetAsync(vb, 0, 4 * nwords, s);
    if (pC->n_blocks > 0) {
        k_tile_mark<<<(unsigned)((pC->n_blocks + 255) / 256), 256, 0, s>>>(
            pC->n_blocks, pC->row.as<int32_t>(), pC->col.as<int32_t>(), gr->g_of.as<int32_t>(),
            gr->h_of.as<int32_t>(), gr->n_h, (uint32_t *)vb);
        cq_count_launch();
    }
    std::vector<uint32_t> bits(nwords);
    cudaMemcpyAsync(bits.data(), vb, 4 * nwords, cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "tile mark")) != CQ_OK) return st;
    std::vector<int2> tiles;
    for (int64_t b = 0; b < nbits; ++b)
        if (bits[b >> 5] & (1u << (b & 31))) tiles.push_back(make_int2((int)(b / gr->n_h), (int)(b % gr->n_h)));
    st_->n_tiles = (int)tiles.size();
    if ((st = cq_alloc(ctx, st_->tiles, sizeof(int2) * (tiles.size() + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, st_->kstart, sizeof(int64_t) * (tiles.size() + 1))) != CQ_OK)
        return st;
    cudaMemcpyAsync(st_->tiles.ptr, tiles.data(), sizeof(int2) * tiles.size(),
                    cudaMemcpyHostToDevice, s);
    const int n_atoms = pA->geo->n_atoms;
    const size_t shm = 2 * 4 * (size_t)((n_atoms + 31) / 32);
    if (shm > 200 * 1024) return cq_fail(ctx, CQ_ERR_INVALID, "split product: too many atoms");
    void *vc;
    if ((st = cq_scratch(ctx, "split_kcnt", 8 * (tiles.size() + 1), &vc)) != CQ_OK) return st;
    if (!tiles.empty()) {
        cudaFuncSetAttribute(k_tile_klist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        cudaFuncSetAttribute(k_tile_klist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        k_tile_klist<false><<<st_->n_tiles, 256, shm, s>>>(
            n_atoms, st_->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
            gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
            pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), (int64_t *)vc, nullptr, nullptr);
        cq_count_launch();
    }
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, st_->kstart.as<int64_t>(), st_->n_tiles)) != CQ_OK)
        return st;
    cudaMemcpyAsync(&st_->n_k, st_->kstart.as<int64_t>() + st_->n_tiles, 8, cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "k lists")) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, st_->klist, 4 * (st_->n_k + 1))) != CQ_OK) return st;
    {
        std::vector<int64_t> ks(st_->n_tiles + 1);
        cudaMemcpyAsync(ks.data(), st_->kstart.ptr, 8 * ks.size(), cudaMemcpyDeviceToHost, s);
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "k lists")) != CQ_OK) return st;
        double chunks = 0.0;
        for (int q = 0; q < st_->n_tiles; ++q)
            chunks += (double)((ks[q + 1] - ks[q] + gr->ca - 1) / gr->ca);
        st_->mma_flops = chunks * 6.0 * KSTEPS * 2.0 * MT * NT * 16;
    }
    if (!tiles.empty()) {
        k_tile_klist<true><<<st_->n_tiles, 256, shm, s>>>(
            n_atoms, st_->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
            gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
            pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), nullptr, st_->kstart.as<int64_t>(),
            st_->klist.as<int32_t>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "k lists")) != CQ_OK) return st;
    const int w = gr->gi + gr->gj;
    if ((st = cq_alloc(ctx, st_->table, 4 * (size_t)(st_->n_k + 1) * w)) != CQ_OK) return st;
    if (!tiles.empty()) {
        k_tile_index<<<st_->n_tiles, 256, 0, s>>>(
            st_->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
            gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
            pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), pB->transpose.as<int64_t>(),
            st_->kstart.as<int64_t>(), st_->klist.as<int32_t>(), st_->table.as<int32_t>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "tile index")) != CQ_OK) return st;
    *out = st_.get();
    ctx->aux[key] = st_;
    return CQ_OK;
}

}  // namespace

cq_status cq_bsmm_split(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                        const double *A, const cq_pattern *pB, const double *B, double beta,
                        const cq_pattern *pC, double *C)
{
    const int nb = pC->geo->uniform_nb;
    if (nb != 9 && nb != 4)
        return cq_fail(ctx, CQ_ERR_INVALID,
                       "split-BF16 product: needs a uniform basis of 4 or 9 orbitals per atom");
    if (pC->n_blocks == 0) return CQ_OK;
    cudaStream_t s = ctx->stream;
    Groups *gr;
    SplitTiles *tiles;
    cq_status st = get_groups(ctx, pC, &gr);
    if (st != CQ_OK) return st;
    if ((st = get_tiles(ctx, pA, pB, pC, gr, &tiles)) != CQ_OK) return st;
    // operands in split form: per plane a main array (8 values per block row, nb = 9) and a
    // tail array (4 values per block row)
    const int mainw = nb == 9 ? KLayout<9>::MAINW : KLayout<4>::MAINW;
    const int ka = mainw + TAILW;
    const int64_t ra = pA->n_blocks * nb, rb = pB->n_blocks * nb;  // block rows
    void *va, *vb;
    if ((st = cq_scratch(ctx, "split_A", 3 * 2 * (size_t)(ra * ka), &va)) != CQ_OK) return st;
    if ((st = cq_scratch(ctx, "split_B", 3 * 2 * (size_t)(rb * ka), &vb)) != CQ_OK) return st;
    SplitPlanes pa, pb;
    {
        __nv_bfloat16 *x = (__nv_bfloat16 *)va, *y = (__nv_bfloat16 *)vb;
        for (int q = 0; q < 3; ++q) {
            pa.main[q] = x + q * ra * mainw;
            pb.main[q] = y + q * rb * mainw;
        }
        for (int q = 0; q < 3; ++q) {
            pa.tail[q] = x + 3 * ra * mainw + q * ra * TAILW;
            pb.tail[q] = y + 3 * rb * mainw + q * rb * TAILW;
        }
    }
    if (ra > 0)
        k_split_a<<<(unsigned)((ra * ka + 255) / 256), 256, 0, s>>>(ra * ka, nb, mainw,
                                                                   pA->uniform, A, pa);
    if (rb > 0)
        k_split_b<<<(unsigned)((rb * ka + 255) / 256), 256, 0, s>>>(rb * ka, nb, mainw,
                                                                   pB->uniform, B, pb);
    cq_count_launch((ra > 0) + (rb > 0));
    SplitArgs a;
    a.n_tiles = tiles->n_tiles;
    a.tiles = tiles->tiles.as<int2>();
    a.kstart = tiles->kstart.as<int64_t>();
    a.klist = tiles->klist.as<int32_t>();
    a.table = tiles->table.as<int32_t>();
    a.g_atoms = gr->g_atoms.as<int32_t>();
    a.h_atoms = gr->h_atoms.as<int32_t>();
    a.a_rp = pA->row_ptr.as<int64_t>();
    a.b_rp = pB->row_ptr.as<int64_t>();
    a.c_rp = pC->row_ptr.as<int64_t>();
    a.a_col = pA->col.as<int32_t>();
    a.b_col = pB->col.as<int32_t>();
    a.c_col = pC->col.as<int32_t>();
    a.b_tr = pB->transpose.as<int64_t>();
    for (int q = 0; q < 3; ++q) {
        a.sa_main[q] = pa.main[q];
        a.sa_tail[q] = pa.tail[q];
        a.sb_main[q] = pb.main[q];
        a.sb_tail[q] = pb.tail[q];
    }
    a.C = C;
    a.c_stride = pC->uniform;
    a.alpha = alpha;
    a.beta = beta;
    a.flag = ctx->flag.as<int32_t>();
    const int grid = std::min(tiles->n_tiles, ctx->num_sms);
    cq_timing_begin(ctx, tl->flops, tiles->mma_flops);
    static bool attr_set = false;  // once per process (outside any graph capture)
    if (!attr_set) {
        cudaFuncSetAttribute(k_bsmm_split<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        cudaFuncSetAttribute(k_bsmm_split<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        attr_set = true;
    }
    if (nb == 9)
        k_bsmm_split<9><<<grid, ST, SMEM, s>>>(a);
    else
        k_bsmm_split<4><<<grid, ST, SMEM, s>>>(a);
    cq_timing_end(ctx);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "bsmm_split");
}
