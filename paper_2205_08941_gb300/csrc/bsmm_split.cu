// Split-BF16 block-sparse product on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// C <- beta C + alpha mask_{P_C}(A.B) with every FP64 operand value split into three BF16
// terms x ~ x0 + x1 + x2 (about 26 bits; see split3) and the product formed as the six
// cross products A_p B_q with p + q <= 2, accumulated in FP32 in tensor memory.  Every
// DRAIN chunks the FP32 accumulator is drained into a per-thread double-float (hi, lo)
// sum, so FP32 rounding only acts within a drain period; the result is written back in
// FP64.
//
// Local densification.  9x9 blocks do not fit MMA shapes, so atoms are grouped in space
// (Morton order): an M group holds floor(128/nb) atoms (126 rows for nb = 9), an N group
// floor(64/nb) atoms.  A work tile is a pair (M group g, N group h) that holds at least one
// block of P_C; its K atoms are the atoms k with (i, k) in P_A for some i in g and (k, j)
// in P_B for some j in h.  Absent blocks are zero.  Every C block belongs to exactly one
// tile, so there are no atomics.
//
// K layout (one MMA K step = 16 values = two core-matrix columns of 8).  An atom's orbitals
// are split into a main piece of 8 (orbitals 0-7, nb = 9 only) and a tail of nb - 8 (or
// nb) values.  A main K step holds the main pieces of two K atoms of the tile, paired in
// order, so a tile's main steps follow its own K atom set; a tail K step holds the tails
// of one fixed tail group (16 consecutive atoms in Morton order for nb = 9, 4 for nb = 4),
// taken when the tile has a K atom in the group.  A 9-orbital atom thus costs 8 K values
// plus a sixteenth of a tail step.
//
// Pieces.  Before each product the operands are split and packed into pieces that are
// byte-for-byte shared-memory images in the canonical no-swizzle K-major layout (core
// matrix = 8 rows x 16 bytes; the 8-row groups of one core column adjacent, 128 B apart):
// an A main piece per (M group, atom k) with a block of P_A (3 planes x 128 rows x 8 K,
// 6 KB), an A tail piece per (M group, tail group) with a block (3 planes x 2 columns,
// 12 KB), and B pieces per N group likewise (64 rows: 3 KB and 6 KB).  Shared memory holds
// a K step in an 18 KB slot, so every step costs the same; the descriptors of a main step
// reach its second atom's column through the leading byte offset, those of a tail step
// its second column.  The tile kernel moves each piece with one TMA bulk copy; one thread
// issues the MMAs, eight warps drain the accumulators (bsmm_split_kernel.cuh).  A pieces
// are packed in batches of M groups so that their scratch stays below A_PANEL_CAP bytes.
//
// The emulated-FP64 product (bsmm_emu_kernel.cuh) keeps fixed K groups of CA atoms (4 for
// nb = 9, 12 for nb = 4) packed into one panel per (atom group, K group) pair, because its
// scale groups are runs of K groups.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "cq_internal.cuh"
#include "emu_digits.cuh"
#include "split3.cuh"

namespace {

constexpr int ST = 320;                      // threads per CTA (10 warps)
constexpr int MT = 128, NT = 64, KCH = 48;   // tile M, N and K chunk
constexpr int KSTEPS = KCH / 16;             // MMA K steps per chunk
constexpr int TAILW = 4;                     // values in an atom's tail piece
constexpr int A_CHUNK = 3 * MT * KCH * 2;   // 36 KB: three planes of 128 rows x 48 K
constexpr int B_CHUNK = 3 * NT * KCH * 2;   // 18 KB
constexpr int STAGE = A_CHUNK + B_CHUNK;    // one shared-memory stage of the split kernel
constexpr int BAR_BYTES = 256;
constexpr int DRAIN = 4;                     // chunks per FP32 accumulation period
constexpr int NACC = 4;                      // FP32 accumulators in tensor memory
constexpr int TMEM_COLS = NACC * NT;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr size_t A_PANEL_CAP = (size_t)12 << 30;  // scratch bound for one batch of A panels

// Split-product pieces and the shared-memory slots of one stage (KSTEPS K steps).
constexpr int COLB_A = MT * 16, COLB_B = NT * 16;  // one core column: 2 KB (A), 1 KB (B)
constexpr int A_MAIN = 3 * COLB_A;                 // 6 KB: planes x one column
constexpr int B_MAIN = 3 * COLB_B;                 // 3 KB
constexpr int A_TAIL = 2 * A_MAIN;                 // 12 KB: planes x two columns
constexpr int B_TAIL = 2 * B_MAIN;                 // 6 KB
constexpr int A_SLOT = A_TAIL, B_SLOT = B_TAIL;    // a K step's room in a stage
constexpr int B_SLOTS = KSTEPS * A_SLOT;           // stage offset of the B slots
static_assert(KSTEPS * (A_SLOT + B_SLOT) == STAGE, "stage layout");

// Main and tail widths of an atom's K values, and atoms per tail group.
template <int NB> struct KPieces;
template <> struct KPieces<9> { static constexpr int MAINW = 8, TW = 1, TG = 16; };
template <> struct KPieces<4> { static constexpr int MAINW = 0, TW = 4, TG = 4; };

// Atoms per chunk and core-matrix columns of an atom's pieces.
template <int NB> struct KLayout;
template <> struct KLayout<9> {
    static constexpr int CA = 4, MAINW = 8;
    __host__ __device__ static constexpr int main_col(int a) { return a; }
    __host__ __device__ static constexpr int tail_col(int a) { return 4 + (a >> 1); }
};
template <> struct KLayout<4> {
    static constexpr int CA = 12, MAINW = 0;
    __host__ __device__ static constexpr int main_col(int) { return 0; }
    __host__ __device__ static constexpr int tail_col(int a) { return a >> 1; }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (plane, core column, row) in a piece: planes plane_b apart, core columns
// col_b apart, each column the 8-row groups of its rows 128 B apart
__host__ __device__ __forceinline__ uint32_t piece_off(int plane, int plane_b, int col, int col_b,
                                                       int row)
{
    return (uint32_t)(plane * plane_b + col * col_b + (row >> 3) * 128 + (row & 7) * 16);
}

// shared-memory descriptor, no swizzle: lbo bytes between the two K-adjacent core columns
// of a K step, 128 bytes between 8-row groups
__device__ __forceinline__ uint64_t piece_desc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // leading (K) byte offset
    d |= (uint64_t)(128 >> 4) << 32;             // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;                      // descriptor version for tcgen05
    return d;                                    // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(MT >> 4) << 24);

// index of block (row, col) in a pattern, or -1
__device__ __forceinline__ int64_t find_block(const int64_t *rp, const int32_t *cl, int row, int col)
{
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cl[mid] < col)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < rp[row + 1] && cl[lo] == col) ? lo : -1;
}

// ---------------------------------------------------------------- plan kernels

// Tile existence: bit (g, h) for every C block (i, j).
__global__ void k_tile_mark(int64_t n_c, const int32_t *c_row, const int32_t *c_col,
                            const int32_t *g_of, const int32_t *h_of, int n_h, uint32_t *bits)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_c) return;
    const int64_t key = (int64_t)g_of[c_row[b]] * n_h + h_of[c_col[b]];
    atomicOr(&bits[key >> 5], 1u << (key & 31));
}

// Scan of a shared-memory bitmap by a 256-thread CTA: COUNT writes the number of set bits,
// FILL writes their indices in ascending order from out + out0.
template <bool FILL>
__device__ void bitmap_emit(const uint32_t *bits, int words, int64_t *count, int64_t out0,
                            int32_t *out)
{
    __shared__ int scan[256];
    const int per = (words + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
    int mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(bits[w]);
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (!FILL) {
        if (threadIdx.x == blockDim.x - 1) *count = scan[threadIdx.x];
        return;
    }
    int64_t o = out0 + scan[threadIdx.x] - mine;
    for (int w = w0; w < w1; ++w) {
        uint32_t v = bits[w];
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            out[o++] = w * 32 + bit;
        }
    }
}

// K groups of each atom group (one CTA per group): every K group holding a column of a row
// of the group's atoms in pattern (rp, col).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_group_kappa(int gsize, const int32_t *atoms, const int64_t *rp, const int32_t *col,
              const int32_t *kg_of, int n_kappa, int64_t *count, const int64_t *start,
              int32_t *out)
{
    extern __shared__ uint32_t bits[];
    const int words = (n_kappa + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    for (int s = 0; s < gsize; ++s) {
        const int i = atoms[(int64_t)blockIdx.x * gsize + s];
        if (i < 0) continue;
        for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
            const int kk = kg_of[col[e]];
            atomicOr(&bits[kk >> 5], 1u << (kk & 31));
        }
    }
    __syncthreads();
    bitmap_emit<FILL>(bits, words, count + blockIdx.x, FILL ? start[blockIdx.x] : 0, out);
}

// K groups of each tile (one CTA per tile): the groups of the atoms k reachable from the M
// group through P_A and from the N group through P_B (P_B symmetric: (k, j) in P_B <=> k in
// row j).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_tile_kappa(int n_atoms, const int2 *tiles, int gi, int gj, const int32_t *g_atoms,
             const int32_t *h_atoms, const int64_t *a_rp, const int32_t *a_col,
             const int64_t *b_rp, const int32_t *b_col, const int32_t *kg_of, int n_kappa,
             int64_t *count, const int64_t *start, int32_t *out)
{
    extern __shared__ uint32_t bm[];
    const int words = (n_atoms + 31) >> 5, kwords = (n_kappa + 31) >> 5;
    uint32_t *ba = bm, *bb = bm + words, *bk = bm + 2 * words;
    for (int w = threadIdx.x; w < 2 * words + kwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int2 t = tiles[blockIdx.x];
    for (int s = 0; s < gi; ++s) {
        const int i = g_atoms[(int64_t)t.x * gi + s];
        if (i < 0) continue;
        for (int64_t e = a_rp[i] + threadIdx.x; e < a_rp[i + 1]; e += blockDim.x)
            atomicOr(&ba[a_col[e] >> 5], 1u << (a_col[e] & 31));
    }
    for (int s = 0; s < gj; ++s) {
        const int j = h_atoms[(int64_t)t.y * gj + s];
        if (j < 0) continue;
        for (int64_t e = b_rp[j] + threadIdx.x; e < b_rp[j + 1]; e += blockDim.x)
            atomicOr(&bb[b_col[e] >> 5], 1u << (b_col[e] & 31));
    }
    __syncthreads();
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        uint32_t v = ba[w] & bb[w];
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            const int kk = kg_of[w * 32 + bit];
            atomicOr(&bk[kk >> 5], 1u << (kk & 31));
        }
    }
    __syncthreads();
    bitmap_emit<FILL>(bk, kwords, count + blockIdx.x, FILL ? start[blockIdx.x] : 0, out);
}

// Chunk table: for every K group of every tile, the A panel (entry of the M group's list)
// and the B panel (entry of the N group's list).
__global__ void __launch_bounds__(256)
k_tile_chunks(const int2 *tiles, const int64_t *kstart, const int32_t *tile_kappa,
              const int64_t *ga_ptr, const int32_t *ga_kappa, const int64_t *hb_ptr,
              const int32_t *hb_kappa, int2 *chunks)
{
    const int2 t = tiles[blockIdx.x];
    auto pos = [](const int32_t *lst, int64_t lo, int64_t hi, int key) {
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (lst[mid] < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        return lo;
    };
    for (int64_t c = kstart[blockIdx.x] + threadIdx.x; c < kstart[blockIdx.x + 1]; c += blockDim.x) {
        const int kk = tile_kappa[c];
        chunks[c] = make_int2((int)pos(ga_kappa, ga_ptr[t.x], ga_ptr[t.x + 1], kk),
                              (int)pos(hb_kappa, hb_ptr[t.y], hb_ptr[t.y + 1], kk));
    }
}

// position of key in the ascending list lst[lo, hi) (the key is present)
__device__ __forceinline__ int64_t list_pos(const int32_t *lst, int64_t lo, int64_t hi, int key)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (lst[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// K-step table of the split product (one CTA per tile): first the main steps, pairing the
// tile's K atoms (Morton ranks, ascending) two by two -- (A main entry, second A main entry
// or -1, B main entry, second B main entry or -1) -- then one tail step per tail group the
// tile touches -- (A tail entry, -1, B tail entry, -1).  Entries index the M group's and
// N group's piece lists.
__global__ void __launch_bounds__(256)
k_tile_steps(const int2 *tiles, const int64_t *ka_start, const int32_t *tile_rank,
             const int64_t *kt_start, const int32_t *tile_tau, const int64_t *step_start,
             const int64_t *gm_ptr, const int32_t *gm_key, const int64_t *hm_ptr,
             const int32_t *hm_key, const int64_t *gt_ptr, const int32_t *gt_key,
             const int64_t *ht_ptr, const int32_t *ht_key, int4 *steps)
{
    const int2 t = tiles[blockIdx.x];
    const int64_t a0 = ka_start[blockIdx.x], na = ka_start[blockIdx.x + 1] - a0;
    const int64_t t0 = kt_start[blockIdx.x], nt = kt_start[blockIdx.x + 1] - t0;
    const int64_t nm = (na + 1) / 2, s0 = step_start[blockIdx.x];
    for (int64_t q = threadIdx.x; q < nm; q += blockDim.x) {
        const int k0 = tile_rank[a0 + 2 * q];
        const int k1 = 2 * q + 1 < na ? tile_rank[a0 + 2 * q + 1] : -1;
        int4 e;
        e.x = (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k0);
        e.y = k1 < 0 ? -1 : (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k1);
        e.z = (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k0);
        e.w = k1 < 0 ? -1 : (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k1);
        steps[s0 + q] = e;
    }
    for (int64_t q = threadIdx.x; q < nt; q += blockDim.x) {
        const int tau = tile_tau[t0 + q];
        steps[s0 + nm + q] = make_int4((int)list_pos(gt_key, gt_ptr[t.x], gt_ptr[t.x + 1], tau), -1,
                                       (int)list_pos(ht_key, ht_ptr[t.y], ht_ptr[t.y + 1], tau), -1);
    }
}

// C block of every (M slot, N slot) pair of each tile: index into P_C or -1, so that the
// epilogue needs one independent load per block instead of a binary search.
__global__ void __launch_bounds__(256)
k_tile_cidx(const int2 *tiles, int gi, int gj, const int32_t *g_atoms, const int32_t *h_atoms,
            const int64_t *c_rp, const int32_t *c_col, int32_t *cidx)
{
    const int2 t = tiles[blockIdx.x];
    for (int e = threadIdx.x; e < gi * gj; e += blockDim.x) {
        const int si = e / gj, sj = e % gj;
        const int i = g_atoms[(int64_t)t.x * gi + si], j = h_atoms[(int64_t)t.y * gj + sj];
        cidx[(int64_t)blockIdx.x * gi * gj + e] =
            (i >= 0 && j >= 0) ? (int32_t)find_block(c_rp, c_col, i, j) : -1;
    }
}

// ---------------------------------------------------------------- panel packing

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Three BF16 planes of eight values x[0..7] (split3), stored as one 16-byte core-matrix
// row per plane at offsets off + plane * plane_b.
__device__ __forceinline__ void put_row3(uint8_t *dst, uint32_t off, int plane_b,
                                         const double (&x)[8])
{
    __nv_bfloat16 v[3][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) split3(x[m], v[0][m], v[1][m], v[2][m]);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        uint4 w;
        w.x = pack_bf16x2(v[pl][0], v[pl][1]);
        w.y = pack_bf16x2(v[pl][2], v[pl][3]);
        w.z = pack_bf16x2(v[pl][4], v[pl][5]);
        w.w = pack_bf16x2(v[pl][6], v[pl][7]);
        *reinterpret_cast<uint4 *>(dst + off + pl * plane_b) = w;
    }
}

// Block index of every (slot, K-group atom) pair of every panel entry (one CTA per entry):
// A side (LEFT): block (i_slot, k) of P_A; B side: block (k, j_slot) of P_B, found as
// block (j, k) of row j and its transpose.  -1 where the pattern has no block.  Patterns
// do not change between products, so the table is built once per pattern triple.
template <bool LEFT>
__global__ void __launch_bounds__(256)
k_panel_index(int gsize, int ca, const int32_t *ent_group, const int32_t *ent_kappa,
              const int32_t *atoms, const int32_t *kg_atoms, const int64_t *rp,
              const int32_t *col, const int64_t *tr, int32_t *index)
{
    const int64_t e = blockIdx.x;
    const int grp = ent_group[e], kk = ent_kappa[e];
    for (int q = threadIdx.x; q < gsize * ca; q += blockDim.x) {
        const int x = atoms[(int64_t)grp * gsize + q / ca], k = kg_atoms[(int64_t)kk * ca + q % ca];
        int64_t b = (x >= 0 && k >= 0) ? find_block(rp, col, x, k) : -1;
        if (!LEFT && b >= 0) b = tr[b];
        index[e * gsize * ca + q] = (int32_t)b;
    }
}

// Main pieces of entries [e0, e0 + n) (one thread per (entry, row)), entry = (atom group,
// K atom k), index = its block per slot (k_panel_index with one atom per K group).  A side
// (LEFT): row r = (slot r / NB, orbital o), K = orbital m < 8 of k: A_ik[o][m]; B side: row
// r = (slot, orbital o of j), K = m: B_kj[m][o].
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_main(int64_t e0, int64_t n, const int32_t *index, const double *__restrict__ X,
            int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS;
    const int r = (int)(q % ROWS), o = r % NB;
    const int64_t b = r < G * NB ? __ldg(&index[(e0 + el) * G + r / NB]) : -1;
    double x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
        x[m] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
    put_row3(pieces + el * (3 * COLB), piece_off(0, COLB, 0, 0, r), COLB, x);
}

// Tail pieces of entries [e0, e0 + n) (one thread per (entry, row)), entry = (atom group,
// tail group), index = its block per (slot, atom u of the tail group).  K position
// u * TW + m (two core columns) = orbital MAINW + m of atom u.
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_tail(int64_t e0, int64_t n, const int32_t *index, const double *__restrict__ X,
            int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    constexpr int MW = KPieces<NB>::MAINW, TW = KPieces<NB>::TW, TG = KPieces<NB>::TG;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS;
    const int r = (int)(q % ROWS), o = r % NB;
    const int32_t *blk = index + ((e0 + el) * G + (r < G * NB ? r / NB : 0)) * TG;
    uint8_t *piece = pieces + el * (6 * COLB);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        double x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int pos = 8 * c + v, u = pos / TW, m = MW + pos % TW;
            const int64_t b = r < G * NB ? __ldg(&blk[u]) : -1;
            x[v] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
        }
        put_row3(piece, piece_off(0, 2 * COLB, c, COLB, r), 2 * COLB, x);
    }
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
    int n_tiles;              // tiles of this launch
    const int64_t *kstart;    // K-step range of each tile (n_tiles + 1, into steps)
    const int32_t *nmain;     // main K steps of each tile (they come first)
    const int4 *steps;        // piece entries of every K step (k_tile_steps)
    const int32_t *cidx;      // C block of each (M slot, N slot) pair of each tile
    const uint8_t *a_main;    // A main pieces of entries [am0, ...)
    int64_t am0;
    const uint8_t *a_tail;    // A tail pieces of entries [at0, ...)
    int64_t at0;
    const uint8_t *b_main;    // all B main pieces
    const uint8_t *b_tail;    // all B tail pieces
    const uint8_t *zero;      // an all-zero A main piece (stands for a missing second atom)
    double *C;
    int c_stride;
    double alpha, beta;
    int32_t *flag;
    long long test_wait_cycles;  // > 0: test mode, the MMA thread's first wait runs out
};

#include "bsmm_split_kernel.cuh"
#include "bsmm_emu_kernel.cuh"

constexpr int SMEM = NS * STAGE + BAR_BYTES;     // pipeline stages + barriers
constexpr int SMEM_E = NSE * E_STAGE + E_LWORDS + BAR_BYTES;

// ---------------------------------------------------------------- emulated-FP64 packing

// Byte offset of (row, core-matrix column col of the chunk's K layout, digit plane) in an
// emulated-FP64 panel: K step col / 2, then the plane, then the canonical no-swizzle
// K-major image of rows x 16 K (core matrices adjacent along K, 8-row groups 256 B apart).
__device__ __forceinline__ uint32_t emu_off(int rows, int row, int col, int plane)
{
    return (uint32_t)((col >> 1) * EMU_P * rows * 32 + plane * rows * 32 + (row >> 3) * E_SBO +
                      (col & 1) * 128 + (row & 7) * 16);
}

// Scale-period flags of every chunk (one CTA per tile): a period is a run of a tile's
// chunks whose K groups share a scale group (K group >> 2).
__global__ void __launch_bounds__(256)
k_emu_periods(const int64_t *kstart, const int32_t *kappa, uint8_t *meta)
{
    const int64_t c0 = kstart[blockIdx.x], c1 = kstart[blockIdx.x + 1];
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const int sg = kappa[c] >> 2;
        uint8_t f = 0;
        if (c == c0 || (kappa[c - 1] >> 2) != sg) f |= 1;
        if (c == c1 - 1 || (kappa[c + 1] >> 2) != sg) f |= 2;
        meta[c] = f;
    }
}

// Largest exponent (emu_exponent) of every scalar row of every A panel entry (one CTA
// of 128 threads per entry = (M group, K group)): row r = (slot r / NB, orbital r % NB).
template <int NB>
__global__ void __launch_bounds__(MT)
k_emu_rowexp_a(const int32_t *index, const double *__restrict__ A, int stride, int16_t *out)
{
    constexpr int GI = MT / NB, CA = KLayout<NB>::CA;
    const int64_t e = blockIdx.x;
    const int r = threadIdx.x;
    int m = EMU_NONE;
    if (r < GI * NB) {
        const int32_t *blk = index + e * (GI * CA) + (r / NB) * CA;
        const int o = r % NB;
        for (int a = 0; a < CA; ++a) {
            const int64_t b = __ldg(&blk[a]);
            if (b < 0) continue;
            for (int k = 0; k < NB; ++k) m = max(m, emu_exponent(A[b * stride + o * NB + k]));
        }
    }
    out[e * MT + r] = (int16_t)m;
}

// The same for every scalar column of every B panel entry (one CTA of 64 threads per entry
// = (N group, K group)): column c = (slot c / NB, orbital o); values B_kj[m][o].
template <int NB>
__global__ void __launch_bounds__(NT)
k_emu_rowexp_b(const int32_t *index, const double *__restrict__ B, int stride, int16_t *out)
{
    constexpr int GJ = NT / NB, CA = KLayout<NB>::CA;
    const int64_t e = blockIdx.x;
    const int c = threadIdx.x;
    int m = EMU_NONE;
    if (c < GJ * NB) {
        const int32_t *blk = index + e * (GJ * CA) + (c / NB) * CA;
        const int o = c % NB;
        for (int a = 0; a < CA; ++a) {
            const int64_t b = __ldg(&blk[a]);
            if (b < 0) continue;
            for (int k = 0; k < NB; ++k) m = max(m, emu_exponent(B[b * stride + k * NB + o]));
        }
    }
    out[e * NT + c] = (int16_t)m;
}

// Group exponent of every (entry, row): the largest row exponent over the entries of the
// same atom group whose K groups share a scale group (K group >> 2).  The entries of a
// group are sorted by K group, so those entries are adjacent.
__global__ void k_emu_group_scale(int width, const int64_t *ptr, const int32_t *kappa,
                                  const int32_t *group, const int16_t *rowexp, int16_t *scale)
{
    const int64_t e = blockIdx.x;
    const int r = threadIdx.x;
    const int g = group[e], sg = kappa[e] >> 2;
    int64_t lo = e, hi = e + 1;
    while (lo > ptr[g] && (kappa[lo - 1] >> 2) == sg) --lo;
    while (hi < ptr[g + 1] && (kappa[hi] >> 2) == sg) ++hi;
    int m = EMU_NONE;
    for (int64_t f = lo; f < hi; ++f) m = max(m, (int)rowexp[f * width + r]);
    scale[e * width + r] = (int16_t)m;
}

// Eight digit planes of n (<= 8) values as eight 16-byte core-matrix rows (one per plane,
// two BF16 per word, values beyond n zero).
__device__ __forceinline__ void emu_rows(const double *x, int n, int E, uint4 (&w)[EMU_P])
{
    uint32_t u[EMU_P][4];
#pragma unroll
    for (int p = 0; p < EMU_P; ++p)
#pragma unroll
        for (int k = 0; k < 4; ++k) u[p][k] = 0u;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (v >= n) break;
        __nv_bfloat16 d[EMU_P];
        emu_digits(x[v], E, d);
#pragma unroll
        for (int p = 0; p < EMU_P; ++p)
            u[p][v >> 1] |= (uint32_t)__bfloat16_as_ushort(d[p]) << (16 * (v & 1));
    }
#pragma unroll
    for (int p = 0; p < EMU_P; ++p) w[p] = make_uint4(u[p][0], u[p][1], u[p][2], u[p][3]);
}

// One row of the K pieces of a pair of atoms (a0 even, a0 + 1) of an emulated panel: the
// two main pieces (8 values each) and the core column the two tails (4 values each) share.
template <int NB>
__device__ __forceinline__ void put_pair_emu(uint8_t *panel, int rows, int r, int a0, int E,
                                             const double (&x0)[KLayout<NB>::MAINW + TAILW],
                                             const double (&x1)[KLayout<NB>::MAINW + TAILW])
{
    constexpr int MW = KLayout<NB>::MAINW;
    uint4 w[EMU_P];
    if (MW) {
        emu_rows(x0, MW, E, w);
#pragma unroll
        for (int p = 0; p < EMU_P; ++p)
            *reinterpret_cast<uint4 *>(panel + emu_off(rows, r, KLayout<NB>::main_col(a0), p)) = w[p];
        emu_rows(x1, MW, E, w);
#pragma unroll
        for (int p = 0; p < EMU_P; ++p)
            *reinterpret_cast<uint4 *>(panel + emu_off(rows, r, KLayout<NB>::main_col(a0 + 1), p)) =
                w[p];
    }
    double t[8];
#pragma unroll
    for (int m = 0; m < TAILW; ++m) {
        t[m] = x0[MW + m];
        t[TAILW + m] = x1[MW + m];
    }
    emu_rows(t, 8, E, w);
#pragma unroll
    for (int p = 0; p < EMU_P; ++p)
        *reinterpret_cast<uint4 *>(panel + emu_off(rows, r, KLayout<NB>::tail_col(a0), p)) = w[p];
}

// Emulated A panels of entries [e0, e0 + gridDim.x): as k_pack_a, eight digit planes per
// value against the (entry, row) group exponent.
template <int NB>
__global__ void __launch_bounds__(256)
k_pack_a_emu(int64_t e0, const int32_t *index, const int16_t *scale, const double *__restrict__ A,
             int stride, uint8_t *panels)
{
    constexpr int GI = MT / NB, CA = KLayout<NB>::CA, KA = KLayout<NB>::MAINW + TAILW;
    const int64_t e = e0 + blockIdx.x;
    const int32_t *blk = index + e * (GI * CA);
    uint8_t *panel = panels + (int64_t)blockIdx.x * E_APANEL;
    for (int q = threadIdx.x; q < MT * (CA / 2); q += blockDim.x) {
        const int a0 = 2 * (q / MT), r = q % MT;
        const bool row = r < GI * NB;
        const int64_t b0 = row ? __ldg(&blk[(r / NB) * CA + a0]) : -1;
        const int64_t b1 = row ? __ldg(&blk[(r / NB) * CA + a0 + 1]) : -1;
        const int E = row ? (int)scale[e * MT + r] : EMU_NONE;
        const int o = r % NB;
        double x0[KA], x1[KA];
#pragma unroll
        for (int m = 0; m < KA; ++m) {
            x0[m] = (b0 >= 0 && m < NB) ? A[b0 * stride + o * NB + m] : 0.0;
            x1[m] = (b1 >= 0 && m < NB) ? A[b1 * stride + o * NB + m] : 0.0;
        }
        put_pair_emu<NB>(panel, MT, r, a0, E, x0, x1);
    }
}

// Emulated B panels (one CTA per entry): row r of the panel = column of C; K = (atom,
// orbital m): B_kj[m][o], against the (entry, column) group exponent.
template <int NB>
__global__ void __launch_bounds__(256)
k_pack_b_emu(const int32_t *index, const int16_t *scale, const double *__restrict__ B, int stride,
             uint8_t *panels)
{
    constexpr int GJ = NT / NB, CA = KLayout<NB>::CA, KA = KLayout<NB>::MAINW + TAILW;
    const int64_t e = blockIdx.x;
    const int32_t *blk = index + e * (GJ * CA);
    uint8_t *panel = panels + e * E_BPANEL;
    for (int q = threadIdx.x; q < NT * (CA / 2); q += blockDim.x) {
        const int a0 = 2 * (q / NT), r = q % NT;
        const bool row = r < GJ * NB;
        const int64_t b0 = row ? __ldg(&blk[(r / NB) * CA + a0]) : -1;
        const int64_t b1 = row ? __ldg(&blk[(r / NB) * CA + a0 + 1]) : -1;
        const int E = row ? (int)scale[e * NT + r] : EMU_NONE;
        const int o = r % NB;
        double x0[KA], x1[KA];
#pragma unroll
        for (int m = 0; m < KA; ++m) {
            x0[m] = (b0 >= 0 && m < NB) ? B[b0 * stride + m * NB + o] : 0.0;
            x1[m] = (b1 >= 0 && m < NB) ? B[b1 * stride + m * NB + o] : 0.0;
        }
        put_pair_emu<NB>(panel, NT, r, a0, E, x0, x1);
    }
}

// ---------------------------------------------------------------- host side

struct Groups {
    int gi = 0, gj = 0, ca = 0;      // atoms per M, N and K group
    int n_g = 0, n_h = 0, n_kappa = 0;
    DevBuf g_atoms, h_atoms, kg_atoms, g_of, h_of, kg_of;
    // split product: K atoms by Morton rank, tail groups of tg consecutive ranks
    int tg = 0, n_tau = 0;
    DevBuf rank_atoms, rank_of, tg_atoms, tg_of;
};

struct Batch {
    int tile0, tile1;   // tiles [tile0, tile1)
    int64_t e0, e1;     // A panel entries [e0, e1)
};

struct SplitPlan {
    int n_tiles = 0;
    int64_t n_chunks = 0, n_ga = 0, n_hb = 0;
    double mma_flops = 0.0;  // tensor-core flops of one product over these tiles
    std::vector<Batch> batches;
    std::vector<int64_t> batch_chunks;
    DevBuf tiles, kstart, tile_kappa, chunks, cidx;
    DevBuf ga_ptr, ga_kappa, ga_group, hb_ptr, hb_kappa, hb_group;
    DevBuf ga_index, hb_index;  // block of every (slot, K-group atom) pair of every entry
    DevBuf meta;                // emulated product: scale-period flags per chunk (on demand)
};

// Piece entries of one operand kind (A or B, main or tail): per atom group, ascending keys
// (Morton ranks or tail groups); index = block of every (slot, atom of the key) pair.
struct PieceList {
    DevBuf ptr, key, group, index;
    std::vector<int64_t> ptr_host;
    int64_t n() const { return ptr_host.empty() ? 0 : ptr_host.back(); }
};

struct PieceBatch {
    int tile0, tile1;        // tiles [tile0, tile1)
    int64_t am0, am1;        // A main entries [am0, am1)
    int64_t at0, at1;        // A tail entries [at0, at1)
};

// Plan of one split product (pattern triple): tiles, K-step table, piece lists.
struct PiecePlan {
    int n_tiles = 0;
    int64_t n_steps = 0;
    double mma_flops = 0.0;  // tensor-core flops of one product over these tiles
    std::vector<PieceBatch> batches;
    std::vector<int64_t> batch_steps;
    DevBuf tiles, kstart, nmain, steps, cidx, zero;
    PieceList am, at, bm, bt;
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

cq_status upload(cq_ctx *ctx, DevBuf &buf, const void *host, size_t bytes)
{
    cq_status st = cq_alloc(ctx, buf, bytes ? bytes : 4);
    if (st != CQ_OK) return st;
    if (bytes)
        st = cq_check_cuda(ctx, cudaMemcpyAsync(buf.ptr, host, bytes, cudaMemcpyHostToDevice,
                                                ctx->stream), "upload");
    return st;
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
    gr->n_kappa = (g.n_atoms + gr->ca - 1) / gr->ca;
    std::vector<int32_t> order = spatial_order(g);
    std::vector<int32_t> ga((size_t)gr->n_g * gr->gi, -1), ha((size_t)gr->n_h * gr->gj, -1),
        ka((size_t)gr->n_kappa * gr->ca, -1);
    gr->tg = nb == 9 ? KPieces<9>::TG : KPieces<4>::TG;
    gr->n_tau = (g.n_atoms + gr->tg - 1) / gr->tg;
    std::vector<int32_t> ta((size_t)gr->n_tau * gr->tg, -1);
    std::vector<int32_t> gof(g.n_atoms), hof(g.n_atoms), kof(g.n_atoms), rof(g.n_atoms),
        tof(g.n_atoms);
    for (int r = 0; r < g.n_atoms; ++r) {
        ga[r] = ha[r] = ka[r] = ta[r] = order[r];
        gof[order[r]] = r / gr->gi;
        hof[order[r]] = r / gr->gj;
        kof[order[r]] = r / gr->ca;
        rof[order[r]] = r;
        tof[order[r]] = r / gr->tg;
    }
    cq_status st;
    if ((st = upload(ctx, gr->g_atoms, ga.data(), 4 * ga.size())) != CQ_OK ||
        (st = upload(ctx, gr->h_atoms, ha.data(), 4 * ha.size())) != CQ_OK ||
        (st = upload(ctx, gr->kg_atoms, ka.data(), 4 * ka.size())) != CQ_OK ||
        (st = upload(ctx, gr->g_of, gof.data(), 4 * gof.size())) != CQ_OK ||
        (st = upload(ctx, gr->h_of, hof.data(), 4 * hof.size())) != CQ_OK ||
        (st = upload(ctx, gr->kg_of, kof.data(), 4 * kof.size())) != CQ_OK ||
        (st = upload(ctx, gr->rank_atoms, order.data(), 4 * order.size())) != CQ_OK ||
        (st = upload(ctx, gr->rank_of, rof.data(), 4 * rof.size())) != CQ_OK ||
        (st = upload(ctx, gr->tg_atoms, ta.data(), 4 * ta.size())) != CQ_OK ||
        (st = upload(ctx, gr->tg_of, tof.data(), 4 * tof.size())) != CQ_OK)
        return st;
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "groups")) != CQ_OK) return st;
    *out = gr.get();
    ctx->aux[key] = gr;
    return CQ_OK;
}

// Key lists of n_groups atom groups in a pattern, key_of mapping an atom to one of n_keys
// keys (its K group, Morton rank or tail group): every key of a column of a row of the
// group's atoms.  ptr (n_groups + 1), kappa (ascending per group), group (entry -> group);
// ptr_host receives ptr.
cq_status group_lists(cq_ctx *ctx, int n_groups, int gsize, const int32_t *atoms,
                      const cq_pattern *p, const int32_t *key_of, int n_keys, DevBuf &ptr,
                      DevBuf &kappa, DevBuf &group, std::vector<int64_t> &ptr_host)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    void *vc;
    if ((st = cq_scratch(ctx, "split_cnt", 8 * ((size_t)n_groups + 1), &vc)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, ptr, 8 * ((size_t)n_groups + 1))) != CQ_OK) return st;
    const size_t shm = 4 * (size_t)((n_keys + 31) / 32);
    cudaFuncSetAttribute(k_group_kappa<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_group_kappa<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_group_kappa<false><<<n_groups, 256, shm, s>>>(gsize, atoms, p->row_ptr.as<int64_t>(),
                                                    p->col.as<int32_t>(), key_of, n_keys,
                                                    (int64_t *)vc, nullptr, nullptr);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, ptr.as<int64_t>(), n_groups)) != CQ_OK) return st;
    ptr_host.assign((size_t)n_groups + 1, 0);
    cudaMemcpyAsync(ptr_host.data(), ptr.ptr, 8 * ptr_host.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "group lists")) != CQ_OK) return st;
    const int64_t n = ptr_host[n_groups];
    if ((st = cq_alloc(ctx, kappa, 4 * (size_t)(n + 1))) != CQ_OK) return st;
    k_group_kappa<true><<<n_groups, 256, shm, s>>>(gsize, atoms, p->row_ptr.as<int64_t>(),
                                                   p->col.as<int32_t>(), key_of, n_keys, nullptr,
                                                   ptr.as<int64_t>(), kappa.as<int32_t>());
    cq_count_launch();
    std::vector<int32_t> grp((size_t)n);
    for (int q = 0; q < n_groups; ++q)
        for (int64_t e = ptr_host[q]; e < ptr_host[q + 1]; ++e) grp[e] = q;
    if ((st = upload(ctx, group, grp.data(), 4 * grp.size())) != CQ_OK) return st;
    return cq_check_cuda(ctx, cudaStreamSynchronize(s), "group lists");
}

// Work tiles of a product, sorted by (g, h): the (M group, N group) pairs that hold a
// block of P_C.
cq_status tile_list(cq_ctx *ctx, const cq_pattern *pC, const Groups *gr, std::vector<int2> &tiles)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    const int64_t nbits = (int64_t)gr->n_g * gr->n_h;
    const int64_t nwords = (nbits + 31) / 32;
    void *vb;
    if ((st = cq_scratch(ctx, "split_bits", 4 * nwords, &vb)) != CQ_OK) return st;
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
    tiles.clear();
    for (int64_t b = 0; b < nbits; ++b)
        if (bits[b >> 5] & (1u << (b & 31)))
            tiles.push_back(make_int2((int)(b / gr->n_h), (int)(b % gr->n_h)));
    return CQ_OK;
}

cq_status get_plan(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                   const cq_pattern *pC, const Groups *gr, SplitPlan **out)
{
    auto key = std::make_tuple(2, pA->id, pB->id, pC->id);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<SplitPlan *>(it->second.get());
        return CQ_OK;
    }
    cudaStream_t s = ctx->stream;
    auto pl = std::make_shared<SplitPlan>();
    cq_status st;
    std::vector<int2> tiles;
    if ((st = tile_list(ctx, pC, gr, tiles)) != CQ_OK) return st;
    pl->n_tiles = (int)tiles.size();
    // K-group lists of the M groups (rows of P_A) and of the N groups (rows of P_B)
    std::vector<int64_t> ga_host, hb_host;
    if ((st = group_lists(ctx, gr->n_g, gr->gi, gr->g_atoms.as<int32_t>(), pA,
                          gr->kg_of.as<int32_t>(), gr->n_kappa, pl->ga_ptr, pl->ga_kappa,
                          pl->ga_group, ga_host)) != CQ_OK ||
        (st = group_lists(ctx, gr->n_h, gr->gj, gr->h_atoms.as<int32_t>(), pB,
                          gr->kg_of.as<int32_t>(), gr->n_kappa, pl->hb_ptr, pl->hb_kappa,
                          pl->hb_group, hb_host)) != CQ_OK)
        return st;
    // batches of whole M groups (tiles are sorted by g) whose A panels fit A_PANEL_CAP
    {
        const int64_t cap = std::max<int64_t>(1, (int64_t)(A_PANEL_CAP / A_CHUNK));
        int t0 = 0;
        while (t0 < pl->n_tiles) {
            const int g0 = tiles[t0].x;
            int t1 = t0, g1 = g0;
            while (t1 < pl->n_tiles) {
                const int g = tiles[t1].x;
                if (g != g1) {  // the next M group starts; keep it only if its panels still fit
                    if (ga_host[g + 1] - ga_host[g0] > cap) break;
                    g1 = g;
                }
                ++t1;
            }
            pl->batches.push_back({t0, t1, ga_host[g0], ga_host[g1 + 1]});
            t0 = t1;
        }
    }
    if ((st = upload(ctx, pl->tiles, tiles.data(), sizeof(int2) * tiles.size())) != CQ_OK) return st;
    pl->n_ga = ga_host[gr->n_g];
    pl->n_hb = hb_host[gr->n_h];
    if ((st = cq_alloc(ctx, pl->ga_index, 4 * ((size_t)pl->n_ga * gr->gi * gr->ca + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, pl->hb_index, 4 * ((size_t)pl->n_hb * gr->gj * gr->ca + 1))) != CQ_OK)
        return st;
    if (pl->n_ga > 0) {
        k_panel_index<true><<<(unsigned)pl->n_ga, 256, 0, s>>>(
            gr->gi, gr->ca, pl->ga_group.as<int32_t>(), pl->ga_kappa.as<int32_t>(),
            gr->g_atoms.as<int32_t>(), gr->kg_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(),
            pA->col.as<int32_t>(), nullptr, pl->ga_index.as<int32_t>());
        cq_count_launch();
    }
    if (pl->n_hb > 0) {
        k_panel_index<false><<<(unsigned)pl->n_hb, 256, 0, s>>>(
            gr->gj, gr->ca, pl->hb_group.as<int32_t>(), pl->hb_kappa.as<int32_t>(),
            gr->h_atoms.as<int32_t>(), gr->kg_atoms.as<int32_t>(), pB->row_ptr.as<int64_t>(),
            pB->col.as<int32_t>(), pB->transpose.as<int64_t>(), pl->hb_index.as<int32_t>());
        cq_count_launch();
    }
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "panel index")) != CQ_OK) return st;
    if (tiles.empty()) {
        *out = pl.get();
        ctx->aux[key] = pl;
        return CQ_OK;
    }
    // K groups and chunk table of every tile
    const int n_atoms = pA->geo->n_atoms;
    const size_t shm = 4 * (size_t)(2 * ((n_atoms + 31) / 32) + (gr->n_kappa + 31) / 32);
    if (shm > 200 * 1024) return cq_fail(ctx, CQ_ERR_INVALID, "split product: too many atoms");
    void *vc;
    if ((st = cq_scratch(ctx, "split_cnt", 8 * (tiles.size() + 1), &vc)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, pl->kstart, 8 * (tiles.size() + 1))) != CQ_OK) return st;
    cudaFuncSetAttribute(k_tile_kappa<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_tile_kappa<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_tile_kappa<false><<<pl->n_tiles, 256, shm, s>>>(
        n_atoms, pl->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), gr->kg_of.as<int32_t>(), gr->n_kappa,
        (int64_t *)vc, nullptr, nullptr);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, pl->kstart.as<int64_t>(), pl->n_tiles)) != CQ_OK)
        return st;
    std::vector<int64_t> ks(pl->n_tiles + 1);
    cudaMemcpyAsync(ks.data(), pl->kstart.ptr, 8 * ks.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "tile chunks")) != CQ_OK) return st;
    pl->n_chunks = ks[pl->n_tiles];
    pl->mma_flops = (double)pl->n_chunks * 6.0 * KSTEPS * 2.0 * MT * NT * 16;
    if ((st = cq_alloc(ctx, pl->tile_kappa, 4 * (size_t)(pl->n_chunks + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, pl->chunks, sizeof(int2) * (size_t)(pl->n_chunks + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, pl->cidx, 4 * ((size_t)pl->n_tiles * gr->gi * gr->gj + 1))) != CQ_OK)
        return st;
    k_tile_kappa<true><<<pl->n_tiles, 256, shm, s>>>(
        n_atoms, pl->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), gr->kg_of.as<int32_t>(), gr->n_kappa,
        nullptr, pl->kstart.as<int64_t>(), pl->tile_kappa.as<int32_t>());
    k_tile_chunks<<<pl->n_tiles, 256, 0, s>>>(
        pl->tiles.as<int2>(), pl->kstart.as<int64_t>(), pl->tile_kappa.as<int32_t>(),
        pl->ga_ptr.as<int64_t>(), pl->ga_kappa.as<int32_t>(), pl->hb_ptr.as<int64_t>(),
        pl->hb_kappa.as<int32_t>(), pl->chunks.as<int2>());
    k_tile_cidx<<<pl->n_tiles, 256, 0, s>>>(
        pl->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pC->row_ptr.as<int64_t>(), pC->col.as<int32_t>(),
        pl->cidx.as<int32_t>());
    cq_count_launch(3);
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "split plan")) != CQ_OK) return st;
    for (const Batch &bt : pl->batches) pl->batch_chunks.push_back(ks[bt.tile1] - ks[bt.tile0]);
    *out = pl.get();
    ctx->aux[key] = pl;
    return CQ_OK;
}

// Piece list of one operand kind: the keys of every atom group (group_lists) and the block
// of every (slot, key atom) pair (k_panel_index); ca atoms per key, key_atoms listing them.
template <bool LEFT>
cq_status piece_list(cq_ctx *ctx, int n_groups, int gsize, const int32_t *atoms,
                     const cq_pattern *p, const int32_t *key_of, int n_keys, int ca,
                     const int32_t *key_atoms, PieceList &pl)
{
    cq_status st = group_lists(ctx, n_groups, gsize, atoms, p, key_of, n_keys, pl.ptr, pl.key,
                               pl.group, pl.ptr_host);
    if (st != CQ_OK) return st;
    const int64_t n = pl.n();
    if ((st = cq_alloc(ctx, pl.index, 4 * ((size_t)n * gsize * ca + 1))) != CQ_OK) return st;
    if (n > 0) {
        k_panel_index<LEFT><<<(unsigned)n, 256, 0, ctx->stream>>>(
            gsize, ca, pl.group.as<int32_t>(), pl.key.as<int32_t>(), atoms, key_atoms,
            p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
            LEFT ? nullptr : p->transpose.as<int64_t>(), pl.index.as<int32_t>());
        cq_count_launch();
    }
    return cq_check_cuda(ctx, cudaGetLastError(), "piece index");
}

// Keys of every tile (k_tile_kappa with key_of: Morton ranks or tail groups): start
// (n_tiles + 1) on the device and the host, keys ascending per tile.
cq_status tile_keys(cq_ctx *ctx, const DevBuf &tiles, int n_tiles, const Groups *gr,
                    const cq_pattern *pA, const cq_pattern *pB, const int32_t *key_of, int n_keys,
                    DevBuf &start, DevBuf &keys, std::vector<int64_t> &start_host)
{
    cudaStream_t s = ctx->stream;
    const int n_atoms = pA->geo->n_atoms;
    const size_t shm = 4 * (size_t)(2 * ((n_atoms + 31) / 32) + (n_keys + 31) / 32);
    if (shm > 200 * 1024) return cq_fail(ctx, CQ_ERR_INVALID, "split product: too many atoms");
    cq_status st;
    void *vc;
    if ((st = cq_scratch(ctx, "split_cnt", 8 * ((size_t)n_tiles + 1), &vc)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, start, 8 * ((size_t)n_tiles + 1))) != CQ_OK) return st;
    cudaFuncSetAttribute(k_tile_kappa<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_tile_kappa<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_tile_kappa<false><<<n_tiles, 256, shm, s>>>(
        n_atoms, tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), key_of, n_keys, (int64_t *)vc, nullptr,
        nullptr);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, start.as<int64_t>(), n_tiles)) != CQ_OK) return st;
    start_host.assign((size_t)n_tiles + 1, 0);
    cudaMemcpyAsync(start_host.data(), start.ptr, 8 * start_host.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "tile keys")) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, keys, 4 * (size_t)(start_host[n_tiles] + 1))) != CQ_OK) return st;
    k_tile_kappa<true><<<n_tiles, 256, shm, s>>>(
        n_atoms, tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), key_of, n_keys, nullptr,
        start.as<int64_t>(), keys.as<int32_t>());
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "tile keys");
}

cq_status get_piece_plan(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                         const cq_pattern *pC, const Groups *gr, PiecePlan **out)
{
    auto key = std::make_tuple(3, pA->id, pB->id, pC->id);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<PiecePlan *>(it->second.get());
        return CQ_OK;
    }
    cudaStream_t s = ctx->stream;
    auto pl = std::make_shared<PiecePlan>();
    const bool mains = pC->geo->uniform_nb == 9;
    const int n_atoms = pA->geo->n_atoms;
    cq_status st;
    // piece lists: main pieces per (atom group, K atom), tail pieces per (atom group, tail group)
    if (mains &&
        ((st = piece_list<true>(ctx, gr->n_g, gr->gi, gr->g_atoms.as<int32_t>(), pA,
                                gr->rank_of.as<int32_t>(), n_atoms, 1,
                                gr->rank_atoms.as<int32_t>(), pl->am)) != CQ_OK ||
         (st = piece_list<false>(ctx, gr->n_h, gr->gj, gr->h_atoms.as<int32_t>(), pB,
                                 gr->rank_of.as<int32_t>(), n_atoms, 1,
                                 gr->rank_atoms.as<int32_t>(), pl->bm)) != CQ_OK))
        return st;
    if ((st = piece_list<true>(ctx, gr->n_g, gr->gi, gr->g_atoms.as<int32_t>(), pA,
                               gr->tg_of.as<int32_t>(), gr->n_tau, gr->tg,
                               gr->tg_atoms.as<int32_t>(), pl->at)) != CQ_OK ||
        (st = piece_list<false>(ctx, gr->n_h, gr->gj, gr->h_atoms.as<int32_t>(), pB,
                                gr->tg_of.as<int32_t>(), gr->n_tau, gr->tg,
                                gr->tg_atoms.as<int32_t>(), pl->bt)) != CQ_OK)
        return st;
    if ((st = cq_alloc(ctx, pl->zero, A_MAIN)) != CQ_OK) return st;
    cudaMemsetAsync(pl->zero.ptr, 0, A_MAIN, s);
    std::vector<int2> tiles;
    if ((st = tile_list(ctx, pC, gr, tiles)) != CQ_OK) return st;
    pl->n_tiles = (int)tiles.size();
    if (tiles.empty()) {
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "split plan")) != CQ_OK) return st;
        *out = pl.get();
        ctx->aux[key] = pl;
        return CQ_OK;
    }
    // bytes of the A pieces of M groups [g0, g1]
    auto nm_of = [&](int g) { return mains ? pl->am.ptr_host[g] : (int64_t)0; };
    auto a_bytes = [&](int g0, int g1) {
        return (nm_of(g1 + 1) - nm_of(g0)) * (int64_t)A_MAIN +
               (pl->at.ptr_host[g1 + 1] - pl->at.ptr_host[g0]) * (int64_t)A_TAIL;
    };
    // batches of whole M groups (tiles are sorted by g) whose A pieces fit A_PANEL_CAP
    {
        int t0 = 0;
        while (t0 < pl->n_tiles) {
            const int g0 = tiles[t0].x;
            int t1 = t0, g1 = g0;
            while (t1 < pl->n_tiles) {
                const int g = tiles[t1].x;
                if (g != g1) {  // the next M group starts; keep it only if its pieces still fit
                    if (a_bytes(g0, g) > (int64_t)A_PANEL_CAP) break;
                    g1 = g;
                }
                ++t1;
            }
            pl->batches.push_back({t0, t1, nm_of(g0), nm_of(g1 + 1), pl->at.ptr_host[g0],
                                   pl->at.ptr_host[g1 + 1]});
            t0 = t1;
        }
    }
    if ((st = upload(ctx, pl->tiles, tiles.data(), sizeof(int2) * tiles.size())) != CQ_OK) return st;
    // K atoms and tail groups of every tile (temporaries), then the K-step table
    DevBuf ka_start, tile_rank, kt_start, tile_tau;
    std::vector<int64_t> ka, kt;
    if (mains) {
        if ((st = tile_keys(ctx, pl->tiles, pl->n_tiles, gr, pA, pB, gr->rank_of.as<int32_t>(),
                            n_atoms, ka_start, tile_rank, ka)) != CQ_OK)
            return st;
    } else {
        ka.assign((size_t)pl->n_tiles + 1, 0);
        if ((st = upload(ctx, ka_start, ka.data(), 8 * ka.size())) != CQ_OK ||
            (st = cq_alloc(ctx, tile_rank, 4)) != CQ_OK)
            return st;
    }
    if ((st = tile_keys(ctx, pl->tiles, pl->n_tiles, gr, pA, pB, gr->tg_of.as<int32_t>(),
                        gr->n_tau, kt_start, tile_tau, kt)) != CQ_OK)
        return st;
    std::vector<int64_t> step_start((size_t)pl->n_tiles + 1, 0);
    std::vector<int32_t> nmain((size_t)pl->n_tiles);
    for (int b = 0; b < pl->n_tiles; ++b) {
        const int64_t nm = (ka[b + 1] - ka[b] + 1) / 2, nt = kt[b + 1] - kt[b];
        nmain[b] = (int32_t)nm;
        step_start[b + 1] = step_start[b] + nm + nt;
    }
    pl->n_steps = step_start[pl->n_tiles];
    pl->mma_flops = (double)pl->n_steps * 6.0 * 2.0 * MT * NT * 16;
    for (const PieceBatch &bt : pl->batches)
        pl->batch_steps.push_back(step_start[bt.tile1] - step_start[bt.tile0]);
    if ((st = upload(ctx, pl->kstart, step_start.data(), 8 * step_start.size())) != CQ_OK ||
        (st = upload(ctx, pl->nmain, nmain.data(), 4 * nmain.size())) != CQ_OK ||
        (st = cq_alloc(ctx, pl->steps, sizeof(int4) * (size_t)(pl->n_steps + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, pl->cidx, 4 * ((size_t)pl->n_tiles * gr->gi * gr->gj + 1))) != CQ_OK)
        return st;
    k_tile_steps<<<pl->n_tiles, 256, 0, s>>>(
        pl->tiles.as<int2>(), ka_start.as<int64_t>(), tile_rank.as<int32_t>(),
        kt_start.as<int64_t>(), tile_tau.as<int32_t>(), pl->kstart.as<int64_t>(),
        pl->am.ptr.as<int64_t>(), pl->am.key.as<int32_t>(), pl->bm.ptr.as<int64_t>(),
        pl->bm.key.as<int32_t>(), pl->at.ptr.as<int64_t>(), pl->at.key.as<int32_t>(),
        pl->bt.ptr.as<int64_t>(), pl->bt.key.as<int32_t>(), pl->steps.as<int4>());
    k_tile_cidx<<<pl->n_tiles, 256, 0, s>>>(
        pl->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pC->row_ptr.as<int64_t>(), pC->col.as<int32_t>(),
        pl->cidx.as<int32_t>());
    cq_count_launch(2);
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "split plan")) != CQ_OK) return st;
    // the temporaries are freed on return: let the kernels that read them finish
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "split plan")) != CQ_OK) return st;
    *out = pl.get();
    ctx->aux[key] = pl;
    return CQ_OK;
}

template <int NB>
cq_status run_split(cq_ctx *ctx, const PiecePlan *pl, const Groups *gr, double alpha,
                    const cq_pattern *pA, const double *A, const cq_pattern *pB,
                    const double *B, double beta, const cq_pattern *pC, double *C, double flops)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    size_t am_bytes = 0, at_bytes = 0;
    for (const PieceBatch &b : pl->batches) {
        am_bytes = std::max(am_bytes, (size_t)(b.am1 - b.am0) * A_MAIN);
        at_bytes = std::max(at_bytes, (size_t)(b.at1 - b.at0) * A_TAIL);
    }
    // one spare piece of room at the end of each piece array
    void *vam, *vat, *vbm, *vbt;
    if ((st = cq_scratch(ctx, "split_Am", am_bytes + A_TAIL, &vam)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_At", at_bytes + A_TAIL, &vat)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_Bm", (size_t)pl->bm.n() * B_MAIN + A_TAIL, &vbm)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_Bt", (size_t)pl->bt.n() * B_TAIL + A_TAIL, &vbt)) != CQ_OK)
        return st;
    // the shared-memory limit is a per-device attribute: set it once per device, on the
    // first split product there (which runs eagerly: building its plan synchronises)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cq_fail(ctx, CQ_ERR_INVALID, "split product: device index");
    if (!attr_set[dev]) {
        if ((st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_split<9>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM), "split attribute")) != CQ_OK ||
            (st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_split<4>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM), "split attribute")) != CQ_OK)
            return st;
        attr_set[dev] = true;
    }
    auto blocks = [](int64_t n, int rows) { return (unsigned)((n * rows + 255) / 256); };
    if (pl->bm.n() > 0) {
        k_pack_main<NB, false><<<blocks(pl->bm.n(), NT), 256, 0, s>>>(
            0, pl->bm.n(), pl->bm.index.as<int32_t>(), B, pB->uniform, (uint8_t *)vbm);
        cq_count_launch();
    }
    if (pl->bt.n() > 0) {
        k_pack_tail<NB, false><<<blocks(pl->bt.n(), NT), 256, 0, s>>>(
            0, pl->bt.n(), pl->bt.index.as<int32_t>(), B, pB->uniform, (uint8_t *)vbt);
        cq_count_launch();
    }
    for (size_t q = 0; q < pl->batches.size(); ++q) {
        const PieceBatch &b = pl->batches[q];
        if (b.am1 > b.am0) {
            k_pack_main<NB, true><<<blocks(b.am1 - b.am0, MT), 256, 0, s>>>(
                b.am0, b.am1 - b.am0, pl->am.index.as<int32_t>(), A, pA->uniform, (uint8_t *)vam);
            cq_count_launch();
        }
        if (b.at1 > b.at0) {
            k_pack_tail<NB, true><<<blocks(b.at1 - b.at0, MT), 256, 0, s>>>(
                b.at0, b.at1 - b.at0, pl->at.index.as<int32_t>(), A, pA->uniform, (uint8_t *)vat);
            cq_count_launch();
        }
        SplitArgs a;
        a.n_tiles = b.tile1 - b.tile0;
        a.kstart = pl->kstart.as<int64_t>() + b.tile0;
        a.nmain = pl->nmain.as<int32_t>() + b.tile0;
        a.steps = pl->steps.as<int4>();
        a.cidx = pl->cidx.as<int32_t>() + (int64_t)b.tile0 * gr->gi * gr->gj;
        a.a_main = (const uint8_t *)vam;
        a.am0 = b.am0;
        a.a_tail = (const uint8_t *)vat;
        a.at0 = b.at0;
        a.b_main = (const uint8_t *)vbm;
        a.b_tail = (const uint8_t *)vbt;
        a.zero = pl->zero.as<uint8_t>();
        a.C = C;
        a.c_stride = pC->uniform;
        a.alpha = alpha;
        a.beta = beta;
        a.flag = ctx->flag.as<int32_t>();
        a.test_wait_cycles = ctx->test_wait_cycles;
        // this launch's share of the product's useful and tensor-core flops
        const double share =
            pl->n_steps > 0 ? (double)pl->batch_steps[q] / (double)pl->n_steps : 0.0;
        const int grid = std::min(a.n_tiles, ctx->num_sms);
        cq_timing_begin(ctx, flops * share, pl->mma_flops * share);
        k_bsmm_split<NB><<<grid, ST, SMEM, s>>>(a);
        cq_timing_end(ctx);
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "bsmm_split")) != CQ_OK) return st;
    }
    return CQ_OK;
}

template <int NB>
cq_status run_emu(cq_ctx *ctx, const SplitPlan *pl, const Groups *gr, double alpha,
                  const cq_pattern *pA, const double *A, const cq_pattern *pB, const double *B,
                  double beta, const cq_pattern *pC, double *C, double flops)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    size_t a_bytes = 0;
    for (const Batch &b : pl->batches) a_bytes = std::max(a_bytes, (size_t)(b.e1 - b.e0) * E_APANEL);
    void *va, *vb, *ra, *sa, *rb, *sb;
    if ((st = cq_scratch(ctx, "emu_A", a_bytes, &va)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_B", (size_t)pl->n_hb * E_BPANEL, &vb)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_ra", 2 * (size_t)pl->n_ga * MT + 2, &ra)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_sa", 2 * (size_t)pl->n_ga * MT + 2, &sa)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_rb", 2 * (size_t)pl->n_hb * NT + 2, &rb)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_sb", 2 * (size_t)pl->n_hb * NT + 2, &sb)) != CQ_OK)
        return st;
    // the shared-memory limit is a per-device attribute: set it once per device
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cq_fail(ctx, CQ_ERR_INVALID, "emulated product: device index");
    if (!attr_set[dev]) {
        if ((st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_emu<9>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM_E), "emu attribute")) != CQ_OK ||
            (st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_emu<4>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM_E), "emu attribute")) != CQ_OK)
            return st;
        attr_set[dev] = true;
    }
    // group exponents and digit planes of B, then of A (all entries: a scale group's
    // entries may fall in different packing batches)
    if (pl->n_hb > 0) {
        k_emu_rowexp_b<NB><<<(unsigned)pl->n_hb, NT, 0, s>>>(pl->hb_index.as<int32_t>(), B,
                                                              pB->uniform, (int16_t *)rb);
        k_emu_group_scale<<<(unsigned)pl->n_hb, NT, 0, s>>>(
            NT, pl->hb_ptr.as<int64_t>(), pl->hb_kappa.as<int32_t>(), pl->hb_group.as<int32_t>(),
            (const int16_t *)rb, (int16_t *)sb);
        k_pack_b_emu<NB><<<(unsigned)pl->n_hb, 256, 0, s>>>(
            pl->hb_index.as<int32_t>(), (const int16_t *)sb, B, pB->uniform, (uint8_t *)vb);
        cq_count_launch(3);
    }
    if (pl->n_ga > 0) {
        k_emu_rowexp_a<NB><<<(unsigned)pl->n_ga, MT, 0, s>>>(pl->ga_index.as<int32_t>(), A,
                                                              pA->uniform, (int16_t *)ra);
        k_emu_group_scale<<<(unsigned)pl->n_ga, MT, 0, s>>>(
            MT, pl->ga_ptr.as<int64_t>(), pl->ga_kappa.as<int32_t>(), pl->ga_group.as<int32_t>(),
            (const int16_t *)ra, (int16_t *)sa);
        cq_count_launch(2);
    }
    const double mma_flops = (double)pl->n_chunks * KSTEPS * E_MMAS * 2.0 * MT * NT * 16;
    for (size_t q = 0; q < pl->batches.size(); ++q) {
        const Batch &b = pl->batches[q];
        if (b.e1 > b.e0) {
            k_pack_a_emu<NB><<<(unsigned)(b.e1 - b.e0), 256, 0, s>>>(
                b.e0, pl->ga_index.as<int32_t>(), (const int16_t *)sa, A, pA->uniform,
                (uint8_t *)va);
            cq_count_launch();
        }
        EmuArgs a;
        a.n_tiles = b.tile1 - b.tile0;
        a.kstart = pl->kstart.as<int64_t>() + b.tile0;
        a.chunks = pl->chunks.as<int2>();
        a.meta = pl->meta.as<uint8_t>();
        a.cidx = pl->cidx.as<int32_t>() + (int64_t)b.tile0 * gr->gi * gr->gj;
        a.panel_a = (const uint8_t *)va;
        a.ea0 = b.e0;
        a.panel_b = (const uint8_t *)vb;
        a.scale_a = (const int16_t *)sa;
        a.scale_b = (const int16_t *)sb;
        a.C = C;
        a.c_stride = pC->uniform;
        a.alpha = alpha;
        a.beta = beta;
        a.flag = ctx->flag.as<int32_t>();
        const double share =
            pl->n_chunks > 0 ? (double)pl->batch_chunks[q] / (double)pl->n_chunks : 0.0;
        const int grid = std::min(a.n_tiles, ctx->num_sms);
        cq_timing_begin(ctx, flops * share, mma_flops * share);
        k_bsmm_emu<NB><<<grid, ST, SMEM_E, s>>>(a);
        cq_timing_end(ctx);
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "bsmm_emu")) != CQ_OK) return st;
    }
    return CQ_OK;
}

}  // namespace

cq_status cq_bsmm_emu(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                      const double *A, const cq_pattern *pB, const double *B, double beta,
                      const cq_pattern *pC, double *C)
{
    const int nb = pC->geo->uniform_nb;
    if (nb != 9 && nb != 4)
        return cq_fail(ctx, CQ_ERR_INVALID,
                       "emulated-FP64 product: needs a uniform basis of 4 or 9 orbitals per atom");
    if (pC->n_blocks == 0) return CQ_OK;
    Groups *gr;
    SplitPlan *pl;
    cq_status st = get_groups(ctx, pC, &gr);
    if (st != CQ_OK) return st;
    if ((st = get_plan(ctx, pA, pB, pC, gr, &pl)) != CQ_OK) return st;
    if (pl->n_tiles == 0) return CQ_OK;
    if (!pl->meta.ptr) {  // scale-period flags, built once per pattern triple
        if ((st = cq_alloc(ctx, pl->meta, (size_t)pl->n_chunks + 16)) != CQ_OK) return st;
        k_emu_periods<<<pl->n_tiles, 256, 0, ctx->stream>>>(
            pl->kstart.as<int64_t>(), pl->tile_kappa.as<int32_t>(), pl->meta.as<uint8_t>());
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "emu periods")) != CQ_OK) return st;
    }
    return nb == 9 ? run_emu<9>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops)
                   : run_emu<4>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
}

cq_status cq_bsmm_split(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                        const double *A, const cq_pattern *pB, const double *B, double beta,
                        const cq_pattern *pC, double *C)
{
    const int nb = pC->geo->uniform_nb;
    if (nb != 9 && nb != 4)
        return cq_fail(ctx, CQ_ERR_INVALID,
                       "split-BF16 product: needs a uniform basis of 4 or 9 orbitals per atom");
    if (pC->n_blocks == 0) return CQ_OK;
    Groups *gr;
    PiecePlan *pl;
    cq_status st = get_groups(ctx, pC, &gr);
    if (st != CQ_OK) return st;
    if ((st = get_piece_plan(ctx, pA, pB, pC, gr, &pl)) != CQ_OK) return st;
    if (pl->n_tiles == 0) return CQ_OK;
    return nb == 9 ? run_split<9>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops)
                   : run_split<4>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
}
