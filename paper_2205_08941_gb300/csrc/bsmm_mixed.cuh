// Split-BF16 pieces for bases whose atoms carry different orbital counts (5, 9 and 13 in the
// batched workload; any uniform count other than 4 and 9 also takes this path).  Included by
// bsmm_split.cu after the uniform packers.
//
// Atom groups hold as many consecutive atoms (in the groups' spatial order, never across
// cells of a batch) as fit 128 rows (M) or 64 rows (N), so their slot counts vary; a row
// table per group gives every row its slot, the slot atom's orbital count and the orbital
// (slot << 16 | nb << 8 | orbital; -1 for rows past the group's atoms).  An atom of 8 or
// more orbitals has a main piece (orbitals 0-7); its remaining orbitals, or all of a
// smaller atom's, form its tail.  Tail groups hold consecutive atoms whose tails together
// fill at most 16 K values; a position map per tail group gives each of the 16 positions
// its atom (index in the group) and orbital (u << 8 | orbital; -1 past the tails).  Main
// and tail pieces have the same shared-memory images as in the uniform case, so the tile
// kernel's copies and MMAs are unchanged; only its epilogue maps rows and columns through
// the tables.
constexpr int GI_MIX = 25;  // slots of an M group: 128 rows of atoms of at least 5 orbitals
constexpr int GJ_MIX = 12;  // slots of an N group: 64 rows
constexpr int TG_MIX = 16;  // atoms of a tail group at most

// Main pieces of entries [e0, e0 + n) (one thread per (entry, row)); entry = (atom group,
// K atom of rank ent_key[e]); index = its block per slot.  A side (LEFT): A_ik[o][m] of the
// row's slot atom i; B side: B_kj[m][o].  Blocks are row-major at val_off.
template <bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_main_mixed(int64_t e0, int64_t n, const int32_t *index, const int32_t *ent_group,
                  const int32_t *ent_key, const int32_t *rank_atoms, const int32_t *rows,
                  const int32_t *nb, const int64_t *val_off, const double *__restrict__ X,
                  uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = LEFT ? GI_MIX : GJ_MIX;
    constexpr int COLB = LEFT ? COLB_A : COLB_B;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS, e = e0 + el;
    const int r = (int)(q % ROWS);
    const int32_t tab = __ldg(&rows[(int64_t)ent_group[e] * ROWS + r]);
    double x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = 0.0;
    if (tab >= 0) {
        const int s = tab >> 16, nbs = (tab >> 8) & 255, o = tab & 255;
        const int64_t b = __ldg(&index[e * G + s]);
        if (b >= 0) {
            const double *blk = X + val_off[b];
            const int nbk = nb[rank_atoms[ent_key[e]]];
#pragma unroll
            for (int m = 0; m < 8; ++m) x[m] = LEFT ? blk[o * nbk + m] : blk[m * nbs + o];
        }
    }
    put_row3(pieces + el * (3 * COLB), piece_off(0, COLB, 0, 0, r), COLB, x);
}

// Tail pieces of entries [e0, e0 + n) (one thread per (entry, row)); entry = (atom group,
// tail group ent_key[e]); index = its block per (slot, atom u of the tail group).
template <bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_tail_mixed(int64_t e0, int64_t n, const int32_t *index, const int32_t *ent_group,
                  const int32_t *ent_key, const int32_t *tg_atoms, const int32_t *tg_map,
                  const int32_t *rows, const int32_t *nb, const int64_t *val_off,
                  const double *__restrict__ X, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = LEFT ? GI_MIX : GJ_MIX;
    constexpr int COLB = LEFT ? COLB_A : COLB_B;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS, e = e0 + el;
    const int r = (int)(q % ROWS);
    const int32_t tab = __ldg(&rows[(int64_t)ent_group[e] * ROWS + r]);
    const int tau = ent_key[e];
    uint8_t *piece = pieces + el * (6 * COLB);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        double x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            x[v] = 0.0;
            const int32_t pm = __ldg(&tg_map[(int64_t)tau * TG_MIX + 8 * c + v]);
            if (tab < 0 || pm < 0) continue;
            const int s = tab >> 16, nbs = (tab >> 8) & 255, o = tab & 255;
            const int u = pm >> 8, m = pm & 255;
            const int64_t b = __ldg(&index[(e * G + s) * TG_MIX + u]);
            if (b < 0) continue;
            const double *blk = X + val_off[b];
            const int nbk = nb[tg_atoms[(int64_t)tau * TG_MIX + u]];
            x[v] = LEFT ? blk[o * nbk + m] : blk[m * nbs + o];
        }
        put_row3(piece, piece_off(0, 2 * COLB, c, COLB, r), 2 * COLB, x);
    }
}

// Epilogue of one drain thread of a mixed-basis tile: accumulator row arow of M group g,
// columns 32 * half .. + 31 of N group h; each column whose slot pair has a block of P_C
// gets beta C + alpha (hi + lo) at the block's own offset and row stride.
__device__ __forceinline__ void write_rows_mixed(const SplitArgs &p, int tile, int arow, int half,
                                                 const float (&hi)[32], const float (&lo)[32])
{
    const int2 t = p.tiles[tile];
    const int32_t rt = __ldg(&p.g_row[(int64_t)t.x * MT + arow]);
    if (rt < 0) return;
    const int si = rt >> 16, a = rt & 255;
#pragma unroll
    for (int x = 0; x < 32; ++x) {
        const int32_t ct = __ldg(&p.h_col[(int64_t)t.y * NT + half * 32 + x]);
        if (ct < 0) continue;
        const int sj = ct >> 16, nbj = (ct >> 8) & 255, bo = ct & 255;
        const int32_t blk = __ldg(&p.cidx[((int64_t)tile * GI_MIX + si) * GJ_MIX + sj]);
        if (blk < 0) continue;
        double *dst = p.C + p.c_off[blk] + a * nbj + bo;
        const double v = (double)hi[x] + (double)lo[x];
        *dst = p.beta == 0.0 ? p.alpha * v : p.beta * *dst + p.alpha * v;
    }
}
