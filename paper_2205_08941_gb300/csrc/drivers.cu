// Host drivers: Hotelling inversion, Palser-Manolopoulos start, McWeeny purification and the
// Li-Nunes-Vanderbilt minimisation.  All matrix work runs in the library's kernels; the
// host only does scalar arithmetic between phases (chemical potential, CG coefficients, the
// cubic line search) on FP64 scalars read back from device reductions.
//
// Batches (patterns over several independent cells): every scalar is per cell -- traces,
// dots and Gershgorin bounds are segmented reductions over the cells' contiguous blocks,
// and every update L += alpha_c D uses the cell's own coefficient -- while each block
// product covers all cells in one launch.  A single cell uses the unsegmented kernels.
#include <algorithm>
#include <cmath>

#include "cq_internal.cuh"

namespace {

cq_status same_ctx(cq_ctx *ctx, const cq_pattern *a, const cq_pattern *b)
{
    if (!a || !b) return cq_fail(ctx, CQ_ERR_INVALID, "null pattern");
    if (a->ctx != ctx || b->ctx != ctx) return cq_fail(ctx, CQ_ERR_PATTERN, "pattern of another context");
    if (!cq_same_atoms(a, b)) return cq_fail(ctx, CQ_ERR_PATTERN, "patterns over different atoms");
    return CQ_OK;
}

cq_status bsmm(cq_ctx *ctx, double alpha, const cq_pattern *pA, const double *A,
               const cq_pattern *pB, const double *B, double beta, const cq_pattern *pC,
               double *C, cq_precision prec, double *flops = nullptr)
{
    TaskList *tl = nullptr;
    cq_status st = cq_get_tasks(ctx, pA, pB, pC, &tl);
    if (st != CQ_OK) return st;
    if (flops) *flops += tl->flops;
    if (prec == CQ_FP64) return cq_bsmm_f64(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
    if (prec == CQ_FP64_EMU) return cq_bsmm_emu(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
    return cq_bsmm_split(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
}

#define CQ_TRY(x)                          \
    do {                                   \
        cq_status _st = (x);               \
        if (_st != CQ_OK) return _st;      \
    } while (0)

// Quantity q of a per-cell reduction lands in slots [q*nc, q*nc + nc).
cq_status dot_q(cq_ctx *ctx, const cq_pattern *p, const double *a, const double *b, int q)
{
    const int nc = p->n_cells();
    return nc == 1 ? cq_dot_dev(ctx, p, a, b, q) : cq_dot_seg_dev(ctx, p, a, b, q * nc);
}

cq_status trace_q(cq_ctx *ctx, const cq_pattern *pA, const double *A, const cq_pattern *pB,
                  const double *B, int q)
{
    const int nc = pA->n_cells();
    return nc == 1 ? cq_trace_dev(ctx, pA, A, pB, B, q)
                   : cq_trace_seg_dev(ctx, pA, A, pB, B, q * nc);
}

// nq quantities of nc cells: out[q][c]
cq_status fetch_q(cq_ctx *ctx, int nc, int nq, std::vector<std::vector<double>> &out)
{
    std::vector<double> flat(nq * nc);
    CQ_TRY(cq_fetch(ctx, 0, nq * nc, flat.data()));
    out.assign(nq, std::vector<double>(nc));
    for (int q = 0; q < nq; ++q)
        for (int c = 0; c < nc; ++c) out[q][c] = flat[q * nc + c];
    return CQ_OK;
}

// y <- a_c x + b_c y on every cell of p
cq_status axpby_c(cq_ctx *ctx, const cq_pattern *p, const std::vector<double> &a,
                  const double *x, const std::vector<double> &b, double *y)
{
    if (p->n_cells() == 1) return cq_axpby(ctx, p->n_values, a[0], x, b[0], y);
    return cq_axpby_seg(ctx, p, a.data(), x, b.data(), y);
}

cq_status copy_vals(cq_ctx *ctx, double *dst, const double *src, int64_t n)
{
    return cq_check_cuda(ctx, cudaMemcpyAsync(dst, src, sizeof(double) * n,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "copy");
}

}  // namespace

// ---------------------------------------------------------------- Hotelling

extern "C" cq_status cq_hotelling_init(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                       const cq_pattern *pT, double *T)
{
    if (!ctx || !S || !T) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    const int nc = pS->n_cells();
    if (nc == 1) {
        CQ_TRY(cq_row_bounds_dev(ctx, pS, S, 0));
        double b[3];
        CQ_TRY(cq_fetch(ctx, 0, 3, b));
        if (!(b[2] > 0.0)) return cq_fail(ctx, CQ_ERR_NUMERIC, "hotelling_init: S has a zero row");
        return cq_set_identity(ctx, pT, T, 1.0 / b[2]);
    }
    CQ_TRY(cq_row_bounds_seg_dev(ctx, pS, S, 0));
    std::vector<double> b(3 * nc), inv(nc);
    CQ_TRY(cq_fetch(ctx, 0, 3 * nc, b.data()));
    for (int c = 0; c < nc; ++c) {
        if (!(b[3 * c + 2] > 0.0))
            return cq_fail(ctx, CQ_ERR_NUMERIC, "hotelling_init: S has a zero row");
        inv[c] = 1.0 / b[3 * c + 2];
    }
    return cq_set_identity_seg(ctx, pT, T, inv.data());
}

extern "C" cq_status cq_hotelling_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                       const cq_pattern *pT, double *T, double *resid_host)
{
    if (!ctx || !S || !T) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    cq_pattern *pV = nullptr;
    CQ_TRY(cq_pattern_derived(ctx, pS, 1.0, pS, 1.0, pT, &pV));
    void *v, *w;
    CQ_TRY(cq_scratch(ctx, "hot_V", sizeof(double) * pV->n_values, &v));
    CQ_TRY(cq_scratch(ctx, "hot_W", sizeof(double) * pT->n_values, &w));
    double *V = (double *)v, *W = (double *)w;
    CQ_TRY(bsmm(ctx, 1.0, pS, S, pT, T, 0.0, pV, V, CQ_FP64));
    CQ_TRY(cq_frob2_minus_identity_dev(ctx, pV, V, 0));
    CQ_TRY(bsmm(ctx, 1.0, pT, T, pV, V, 0.0, pT, W, CQ_FP64));
    CQ_TRY(cq_axpby(ctx, pT->n_values, -1.0, W, 2.0, T));
    double r2;
    CQ_TRY(cq_fetch(ctx, 0, 1, &r2));
    if (resid_host) *resid_host = std::sqrt(r2);
    return CQ_OK;
}

// Least-squares overlap inverse: minimise f(T) = ||I - S T||_F^2 over symmetric T on P_T by
// linear conjugate gradients.  R = I - S T is kept on P_V = P_{rS+rT} (the whole residual);
// the gradient on P_T is G = -(W + W^T), W = mask_{P_T}(S R); along D the exact minimiser is
// a = -<G, D> / (2 ||S D||^2); then T += a D, R -= a S D and D <- -G + (<G,G>/<G_prev,G_prev>) D.
extern "C" cq_status cq_overlap_inverse_cg(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                           const cq_pattern *pT, double *T, int32_t max_iter,
                                           double gtol, double *resid_host, double *gnorm_host,
                                           int32_t *iters_host)
{
    if (!ctx || !S || !T || max_iter < 0 || !(gtol >= 0.0)) return CQ_ERR_INVALID;
    if (iters_host) *iters_host = -1;  // no history entry written yet
    CQ_TRY(same_ctx(ctx, pS, pT));
    if (pS->n_cells() != 1 || pT->n_cells() != 1)
        return cq_fail(ctx, CQ_ERR_INVALID, "overlap_inverse_cg: batch patterns not supported");
    cq_pattern *pV = nullptr;
    CQ_TRY(cq_pattern_derived(ctx, pS, 1.0, pS, 1.0, pT, &pV));
    const int64_t nT = pT->n_values, nV = pV->n_values;
    void *r, *sd, *w, *g, *d;
    CQ_TRY(cq_scratch(ctx, "sinv_R", sizeof(double) * nV, &r));
    CQ_TRY(cq_scratch(ctx, "sinv_SD", sizeof(double) * nV, &sd));
    CQ_TRY(cq_scratch(ctx, "sinv_W", sizeof(double) * nT, &w));
    CQ_TRY(cq_scratch(ctx, "sinv_G", sizeof(double) * nT, &g));
    CQ_TRY(cq_scratch(ctx, "sinv_D", sizeof(double) * nT, &d));
    double *R = (double *)r, *SD = (double *)sd, *W = (double *)w, *G = (double *)g,
           *D = (double *)d;
    CQ_TRY(cq_set_identity(ctx, pV, R, 1.0));
    CQ_TRY(bsmm(ctx, -1.0, pS, S, pT, T, 1.0, pV, R, CQ_FP64));  // R = I - S T
    double g0 = 0.0, gg_prev = 0.0;
    int32_t k = 0;
    for (;; ++k) {
        CQ_TRY(bsmm(ctx, 1.0, pS, S, pV, R, 0.0, pT, W, CQ_FP64));
        CQ_TRY(cq_axpby(ctx, nT, -1.0, W, 0.0, G));
        CQ_TRY(cq_gather(ctx, pT, W, pT, G, 1, -1.0, 1.0));      // G = -(W + W^T)
        CQ_TRY(cq_dot_dev(ctx, pT, G, G, 0));
        CQ_TRY(cq_dot_dev(ctx, pV, R, R, 1));
        double v[2];
        CQ_TRY(cq_fetch(ctx, 0, 2, v));
        if (!std::isfinite(v[0]) || !std::isfinite(v[1]))
            return cq_fail(ctx, CQ_ERR_NUMERIC, "overlap_inverse_cg: non-finite residual");
        const double gn = std::sqrt(v[0]);
        if (resid_host) resid_host[k] = std::sqrt(v[1]);
        if (gnorm_host) gnorm_host[k] = gn;
        if (iters_host) *iters_host = k;  // entries 0..k of the histories hold values
        if (k == 0) g0 = gn;
        if (k == max_iter || gn <= gtol * g0) break;
        CQ_TRY(cq_axpby(ctx, nT, -1.0, G, k == 0 ? 0.0 : v[0] / gg_prev, D));
        CQ_TRY(bsmm(ctx, 1.0, pS, S, pT, D, 0.0, pV, SD, CQ_FP64));
        CQ_TRY(cq_dot_dev(ctx, pT, G, D, 0));
        CQ_TRY(cq_dot_dev(ctx, pV, SD, SD, 1));
        double q[2];
        CQ_TRY(cq_fetch(ctx, 0, 2, q));
        if (!(q[1] > 0.0) || !std::isfinite(q[0]))
            return cq_fail(ctx, CQ_ERR_NUMERIC, "overlap_inverse_cg: degenerate direction");
        const double a = -q[0] / (2.0 * q[1]);
        CQ_TRY(cq_axpby(ctx, nT, a, D, 1.0, T));
        CQ_TRY(cq_axpby(ctx, nV, -a, SD, 1.0, R));
        gg_prev = v[0];
    }
    return CQ_OK;
}

// ---------------------------------------------------------------- PM start, McWeeny

extern "C" cq_status cq_pm_guess_cells(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                       const double *H, const cq_pattern *pT, const double *T,
                                       const cq_pattern *pL, double *L,
                                       const double *n_occ_host)
{
    if (!ctx || !S || !H || !T || !L || !n_occ_host) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    CQ_TRY(same_ctx(ctx, pS, pL));
    const int nc = pS->n_cells();
    for (int c = 0; c < nc; ++c) {
        const double n_orb = (double)pS->geo->cell_orb[c];
        if (!(n_occ_host[c] > 0.0 && n_occ_host[c] < n_orb))
            return cq_fail(ctx, CQ_ERR_INVALID, "pm_guess: n_occ outside (0, N)");
    }
    cq_pattern *pX = nullptr;
    CQ_TRY(cq_pattern_derived(ctx, pS, 1.0, pT, 1.0, pS, &pX));
    void *th;
    CQ_TRY(cq_scratch(ctx, "pm_TH", sizeof(double) * pX->n_values, &th));
    double *TH = (double *)th;
    CQ_TRY(bsmm(ctx, 1.0, pT, T, pS, H, 0.0, pX, TH, CQ_FP64));
    if (nc == 1) {
        const double n_orb = (double)pS->geo->n_orb, n_occ = n_occ_host[0];
        CQ_TRY(cq_trace_dev(ctx, pT, T, pS, H, 0));
        CQ_TRY(cq_row_bounds_dev(ctx, pX, TH, 1));
        double sc[4];
        CQ_TRY(cq_fetch(ctx, 0, 4, sc));
        const double mu = sc[0] / n_orb;
        const double h_min = sc[1], h_max = sc[2];
        const double lam = std::fmin(n_occ / (h_max - mu), (n_orb - n_occ) / (mu - h_min));
        CQ_TRY(bsmm(ctx, -lam / n_orb, pX, TH, pT, T, 0.0, pL, L, CQ_FP64));
        return cq_gather(ctx, pT, T, pL, L, 0, lam * mu / n_orb + n_occ / n_orb, 1.0);
    }
    CQ_TRY(cq_trace_seg_dev(ctx, pT, T, pS, H, 0));
    CQ_TRY(cq_row_bounds_seg_dev(ctx, pX, TH, nc));
    std::vector<double> sc(4 * nc);
    CQ_TRY(cq_fetch(ctx, 0, 4 * nc, sc.data()));
    std::vector<double> a(nc), b(nc), one(nc, 1.0), zero(nc, 0.0);
    for (int c = 0; c < nc; ++c) {
        const double n_orb = (double)pS->geo->cell_orb[c], n_occ = n_occ_host[c];
        const double mu = sc[c] / n_orb;
        const double h_min = sc[nc + 3 * c], h_max = sc[nc + 3 * c + 1];
        const double lam = std::fmin(n_occ / (h_max - mu), (n_orb - n_occ) / (mu - h_min));
        a[c] = -lam / n_orb;
        b[c] = lam * mu / n_orb + n_occ / n_orb;
    }
    // L = a_c THT + b_c T on P_L
    CQ_TRY(bsmm(ctx, 1.0, pX, TH, pT, T, 0.0, pL, L, CQ_FP64));
    CQ_TRY(axpby_c(ctx, pL, a, L, zero, L));
    void *tl;
    CQ_TRY(cq_scratch(ctx, "pm_TL", sizeof(double) * pL->n_values, &tl));
    CQ_TRY(cq_gather(ctx, pT, T, pL, (double *)tl, 0, 1.0, 0.0));
    return axpby_c(ctx, pL, b, (double *)tl, one, L);
}

extern "C" cq_status cq_pm_guess(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                 const double *H, const cq_pattern *pT, const double *T,
                                 const cq_pattern *pL, double *L, double n_occ)
{
    if (!ctx || !pS) return CQ_ERR_INVALID;
    if (pS->n_cells() != 1)
        return cq_fail(ctx, CQ_ERR_INVALID, "pm_guess: batch patterns need cq_pm_guess_cells");
    return cq_pm_guess_cells(ctx, pS, S, H, pT, T, pL, L, &n_occ);
}

extern "C" cq_status cq_mcweeny_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                     const cq_pattern *pL, double *L)
{
    if (!ctx || !S || !L) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pL));
    cq_pattern *pX, *pU, *p2L;
    CQ_TRY(cq_pattern_derived(ctx, pS, 1.0, pL, 1.0, pS, &pX));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0, pS, 1.0, pL, &pU));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0, pL, 0.0, pL, &p2L));
    void *x, *u, *m, *o;
    CQ_TRY(cq_scratch(ctx, "mw_X", sizeof(double) * pX->n_values, &x));
    CQ_TRY(cq_scratch(ctx, "mw_U", sizeof(double) * pU->n_values, &u));
    CQ_TRY(cq_scratch(ctx, "mw_M", sizeof(double) * p2L->n_values, &m));
    CQ_TRY(cq_scratch(ctx, "mw_O", sizeof(double) * pL->n_values, &o));
    double *X = (double *)x, *U = (double *)u, *M = (double *)m, *O = (double *)o;
    CQ_TRY(bsmm(ctx, 1.0, pL, L, pS, S, 0.0, pX, X, CQ_FP64));
    CQ_TRY(bsmm(ctx, 1.0, pS, S, pX, X, 0.0, pU, U, CQ_FP64));
    CQ_TRY(bsmm(ctx, 1.0, pL, L, pU, U, 0.0, p2L, M, CQ_FP64));
    CQ_TRY(bsmm(ctx, 3.0, pX, X, pL, L, 0.0, pL, O, CQ_FP64));
    CQ_TRY(bsmm(ctx, -2.0, p2L, M, pL, L, 1.0, pL, O, CQ_FP64));
    return copy_vals(ctx, L, O, pL->n_values);
}

// ---------------------------------------------------------------- LNV

struct cq_lnv {
    cq_ctx *ctx = nullptr;
    const cq_pattern *pS = nullptr, *pL = nullptr;
    cq_pattern *pX = nullptr, *pU = nullptr;
    const double *S = nullptr, *H = nullptr;
    double *L = nullptr;
    int nc = 1;
    std::vector<double> ne, E, N, alpha_prev;
    std::vector<int> n_corr_initial;
    cq_precision prec = CQ_FP64;
    DevBuf X, Y, U, Z, R1, R2, R3, GE, GN, G, Gp, D, Dp, Lt;
    bool have_prev = false, have_alpha = false;
    // optional preconditioner: search directions from Zs = sym(mask_L(T G T))
    bool precond = false;
    const cq_pattern *pT = nullptr;
    cq_pattern *pTL = nullptr;      // reaches r_T + r_L (holds T G)
    DevBuf T, TG, Zr, Zs, Zp;       // copy of T; T G; raw, symmetrised and previous Z
    double n_tol = 1e-10;
    double n_tol_split = 1e-9;
    int max_corr = 5;
    double flops = 0.0;
    int products = 0;
    // CUDA graphs of the evaluation phases, keyed (phase, source L, precision)
    struct Graph {
        bool warm = false;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
        double flops = 0.0;
        int products = 0;
        uint64_t gen = 0;  // context scratch generation at capture
    };
    std::map<std::tuple<int, const void *, int>, Graph> graphs;
    ~cq_lnv()
    {
        for (auto &kv : graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    }
};

namespace {

// Device-only phase `body` (products, traces, gradients; no host synchronisation).  With
// graphs off it runs directly.  With graphs on it runs eagerly the first time (building task
// lists and sizing scratch), is captured into a CUDA graph the second time and replayed
// from then on; the graph's launches, flops and products are credited at every replay.
template <class F>
cq_status run_phase(cq_lnv *s, int phase, const void *key, F body)
{
    cq_ctx *ctx = s->ctx;
    if (!ctx->graphs) return body();
    cq_lnv::Graph &g = s->graphs[std::make_tuple(phase, key, (int)s->prec)];
    if (g.exec && g.gen != ctx->scratch_gen) {
        // a scratch buffer the graph reads was reallocated (or released) since the capture:
        // run eagerly once more (rebuilding what was freed), then capture again
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        g.warm = false;
    }
    if (!g.exec) {
        if (!g.warm || g.gen != ctx->scratch_gen) {
            g.warm = true;
            const cq_status st = body();
            g.gen = ctx->scratch_gen;  // the scratch this eager run left behind
            return st;
        }
        const double f0 = s->flops;
        const int p0 = s->products;
        CQ_TRY(cq_check_cuda(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed),
                             "begin capture"));
        ctx->capturing = true;
        cq_capture_counting(true);
        cq_status st = body();
        cq_capture_counting(false);
        ctx->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        g.launches = cq_capture_launches();
        g.flops = s->flops - f0;
        g.products = s->products - p0;
        s->flops = f0;
        s->products = p0;
        if (st != CQ_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return st != CQ_OK ? st : cq_check_cuda(ctx, e, "end capture");
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CQ_TRY(cq_check_cuda(ctx, e, "graph instantiate"));
        g.gen = ctx->scratch_gen;
    }
    CQ_TRY(cq_check_cuda(ctx, cudaGraphLaunch(g.exec, ctx->stream), "graph launch"));
    cq_count_launch(g.launches);
    s->flops += g.flops;
    s->products += g.products;
    return CQ_OK;
}

// E and N (per cell) at Lsrc from the five products a trial point needs (X, Y, U, R1, R3).
cq_status lnv_energy_number(cq_lnv *s, const double *Lsrc, std::vector<double> &E,
                            std::vector<double> &N)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *Y = s->Y.as<double>(), *U = s->U.as<double>();
    double *R1 = s->R1.as<double>(), *R3 = s->R3.as<double>();
    CQ_TRY(run_phase(s, 1, Lsrc, [&]() -> cq_status {
        CQ_TRY(bsmm(ctx, 1.0, s->pL, Lsrc, s->pS, s->S, 0.0, s->pX, X, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pL, Lsrc, s->pS, s->H, 0.0, s->pX, Y, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, X, 0.0, s->pU, U, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, Y, 0.0, s->pL, R1, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, X, 0.0, s->pL, R3, s->prec, &s->flops));
        s->products += 5;
        CQ_TRY(trace_q(ctx, s->pX, X, s->pX, Y, 0));
        CQ_TRY(trace_q(ctx, s->pL, Lsrc, s->pL, R1, 1));
        CQ_TRY(trace_q(ctx, s->pX, X, s->pX, X, 2));
        return trace_q(ctx, s->pL, Lsrc, s->pL, R3, 3);
    }));
    std::vector<std::vector<double>> t;
    CQ_TRY(fetch_q(ctx, s->nc, 4, t));
    E.resize(s->nc);
    N.resize(s->nc);
    for (int c = 0; c < s->nc; ++c) {
        E[c] = 2.0 * (3.0 * t[0][c] - 2.0 * t[1][c]);
        N[c] = 2.0 * (3.0 * t[2][c] - 2.0 * t[3][c]);
    }
    return CQ_OK;
}

// Electron-number half of an evaluation at s->L: X = LS, U = SX, R3 = UX, N and G_N.
// (The products and values are those of a full evaluation; E and G_E follow in
// lnv_eval_rest at the same L.)
cq_status lnv_eval_n(cq_lnv *s)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *U = s->U.as<double>(), *R3 = s->R3.as<double>();
    CQ_TRY(run_phase(s, 2, s->L, [&]() -> cq_status {
        CQ_TRY(bsmm(ctx, 1.0, s->pL, s->L, s->pS, s->S, 0.0, s->pX, X, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, X, 0.0, s->pU, U, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, X, 0.0, s->pL, R3, s->prec, &s->flops));
        s->products += 3;
        CQ_TRY(trace_q(ctx, s->pX, X, s->pX, X, 0));
        CQ_TRY(trace_q(ctx, s->pL, s->L, s->pL, R3, 1));
        return cq_lnv_gradient_n(ctx, s->pL, s->pU, U, R3, s->GN.as<double>());
    }));
    std::vector<std::vector<double>> t;
    CQ_TRY(fetch_q(ctx, s->nc, 2, t));
    s->N.resize(s->nc);
    for (int c = 0; c < s->nc; ++c) s->N[c] = 2.0 * (3.0 * t[0][c] - 2.0 * t[1][c]);
    return CQ_OK;
}

// Energy half at the L of the last lnv_eval_n (X, U still current): Y = LH, R1 = UY,
// Z = SY, R2 = ZX, E and G_E.
cq_status lnv_eval_rest(cq_lnv *s)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *Y = s->Y.as<double>(), *U = s->U.as<double>();
    double *Z = s->Z.as<double>(), *R1 = s->R1.as<double>(), *R2 = s->R2.as<double>();
    CQ_TRY(run_phase(s, 3, s->L, [&]() -> cq_status {
        CQ_TRY(bsmm(ctx, 1.0, s->pL, s->L, s->pS, s->H, 0.0, s->pX, Y, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, Y, 0.0, s->pL, R1, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, Y, 0.0, s->pU, Z, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pU, Z, s->pX, X, 0.0, s->pL, R2, s->prec, &s->flops));
        s->products += 4;
        CQ_TRY(trace_q(ctx, s->pX, X, s->pX, Y, 0));
        CQ_TRY(trace_q(ctx, s->pL, s->L, s->pL, R1, 1));
        return cq_lnv_gradient_e(ctx, s->pL, s->pU, Z, R1, R2, s->GE.as<double>());
    }));
    std::vector<std::vector<double>> t;
    CQ_TRY(fetch_q(ctx, s->nc, 2, t));
    s->E.resize(s->nc);
    for (int c = 0; c < s->nc; ++c) s->E[c] = 2.0 * (3.0 * t[0][c] - 2.0 * t[1][c]);
    return CQ_OK;
}

// <a, b> per cell
cq_status dots(cq_lnv *s, const double *a, const double *b, std::vector<double> &out)
{
    CQ_TRY(dot_q(s->ctx, s->pL, a, b, 0));
    std::vector<std::vector<double>> t;
    CQ_TRY(fetch_q(s->ctx, s->nc, 1, t));
    out = t[0];
    return CQ_OK;
}

// Evaluate at s->L with the electron-number corrections in between: N and G_N first, then
// L += ((N_e - N)/<G_N,G_N>) G_N (at most max_corr times) while |N - N_e| > n_tol N_e, each
// followed by N and G_N at the corrected L, and finally E and G_E at the last L.  The
// iterates and decisions are those of "full evaluation, then correct and re-evaluate";
// only the E half of the intermediate evaluations (never used) is skipped.  In a batch a
// cell within tolerance receives a zero correction.
cq_status lnv_evaluate_corrected(cq_lnv *s, std::vector<int> &count)
{
    CQ_TRY(lnv_eval_n(s));
    count.assign(s->nc, 0);
    // split-BF16 products resolve N to ~1e-10 relative, so their corrections stop at 1e-9
    const double tol = s->prec == CQ_SPLIT_BF16X3 ? s->n_tol_split : s->n_tol;
    for (int k = 0; k < s->max_corr; ++k) {
        std::vector<bool> need(s->nc);
        bool any = false;
        for (int c = 0; c < s->nc; ++c) {
            need[c] = std::fabs(s->N[c] - s->ne[c]) > tol * s->ne[c];
            any = any || need[c];
        }
        if (!any) break;
        std::vector<double> gn2;
        CQ_TRY(dots(s, s->GN.as<double>(), s->GN.as<double>(), gn2));
        std::vector<double> a(s->nc, 0.0), one(s->nc, 1.0);
        for (int c = 0; c < s->nc; ++c)
            if (need[c]) {
                a[c] = (s->ne[c] - s->N[c]) / gn2[c];
                count[c] += 1;
            }
        CQ_TRY(axpby_c(s->ctx, s->pL, a, s->GN.as<double>(), one, s->L));
        CQ_TRY(lnv_eval_n(s));
    }
    return lnv_eval_rest(s);
}

// mu_c = <G_E,G_N>/<G_N,G_N> and G = G_E - mu_c G_N into s->G; returns <G_N,G_N> per cell.
cq_status lnv_mu_g(cq_lnv *s, std::vector<double> &mu, std::vector<double> &gn2)
{
    cq_ctx *ctx = s->ctx;
    CQ_TRY(dot_q(ctx, s->pL, s->GE.as<double>(), s->GN.as<double>(), 0));
    CQ_TRY(dot_q(ctx, s->pL, s->GN.as<double>(), s->GN.as<double>(), 1));
    std::vector<std::vector<double>> d;
    CQ_TRY(fetch_q(ctx, s->nc, 2, d));
    mu.resize(s->nc);
    gn2 = d[1];
    std::vector<double> neg(s->nc), one(s->nc, 1.0);
    for (int c = 0; c < s->nc; ++c) {
        mu[c] = d[0][c] / d[1][c];
        neg[c] = -mu[c];
    }
    CQ_TRY(copy_vals(ctx, s->G.as<double>(), s->GE.as<double>(), s->pL->n_values));
    return axpby_c(ctx, s->pL, neg, s->GN.as<double>(), one, s->G.as<double>());
}

void cubic_coeffs(double f0, double g, double a1, double f1, double a2, double f2, double *c2,
                  double *c3)
{
    const double r1 = f1 - f0 - g * a1;
    const double r2 = f2 - f0 - g * a2;
    const double det = a1 * a1 * a2 * a2 * (a2 - a1);
    *c2 = (r1 * (a2 * a2 * a2) - r2 * (a1 * a1 * a1)) / det;
    *c3 = (a1 * a1 * r2 - a2 * a2 * r1) / det;
}

bool cubic_min(double w1, double w2, double w3, double *a)
{
    const double disc = 4.0 * w2 * w2 - 12.0 * w3 * w1;
    if (disc < 0.0) return false;
    const double den = 2.0 * w2 + std::sqrt(disc);
    if (den <= 0.0) return false;
    *a = -2.0 * w1 / den;
    return *a > 0.0;
}

cq_status lnv_report(cq_lnv *s, cq_lnv_report *rep)
{
    std::vector<double> mu, gn2, gg;
    CQ_TRY(lnv_mu_g(s, mu, gn2));
    CQ_TRY(dots(s, s->G.as<double>(), s->G.as<double>(), gg));
    for (int c = 0; c < s->nc; ++c) {
        rep[c].energy = s->E[c];
        rep[c].n_elec = s->N[c];
        rep[c].mu = mu[c];
        rep[c].gnorm = std::sqrt(gg[c] / (double)s->pL->seg_scalars[c]);
    }
    return CQ_OK;
}

}  // namespace

extern "C" cq_status cq_lnv_create_cells(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                         const double *H, const cq_pattern *pL, double *L,
                                         const double *n_electrons_host, cq_precision prec,
                                         cq_lnv **out)
{
    if (!ctx || !out || !S || !H || !L || !n_electrons_host) return CQ_ERR_INVALID;
    *out = nullptr;
    CQ_TRY(same_ctx(ctx, pS, pL));
    const int nc = pS->n_cells();
    for (int c = 0; c < nc; ++c)
        if (!(n_electrons_host[c] > 0.0 && n_electrons_host[c] < 2.0 * (double)pS->geo->cell_orb[c]))
            return cq_fail(ctx, CQ_ERR_INVALID, "lnv_create: electron count outside (0, 2N)");
    if (prec != CQ_FP64 && prec != CQ_SPLIT_BF16X3 && prec != CQ_FP64_EMU)
        return cq_fail(ctx, CQ_ERR_INVALID, "lnv_create: unknown precision");
    std::unique_ptr<cq_lnv> s(new cq_lnv());
    s->ctx = ctx;
    s->pS = pS;
    s->pL = pL;
    s->S = S;
    s->H = H;
    s->L = L;
    s->nc = nc;
    s->ne.assign(n_electrons_host, n_electrons_host + nc);
    s->alpha_prev.assign(nc, 0.0);
    s->prec = prec;
    CQ_TRY(cq_pattern_derived(ctx, pS, 1.0, pL, 1.0, pS, &s->pX));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0, pS, 1.0, pL, &s->pU));
    const size_t bx = sizeof(double) * s->pX->n_values, bu = sizeof(double) * s->pU->n_values;
    const size_t bl = sizeof(double) * pL->n_values;
    CQ_TRY(cq_alloc(ctx, s->X, bx));
    CQ_TRY(cq_alloc(ctx, s->Y, bx));
    CQ_TRY(cq_alloc(ctx, s->U, bu));
    CQ_TRY(cq_alloc(ctx, s->Z, bu));
    for (DevBuf *b : {&s->R1, &s->R2, &s->R3, &s->GE, &s->GN, &s->G, &s->Gp, &s->D, &s->Dp, &s->Lt})
        CQ_TRY(cq_alloc(ctx, *b, bl));
    CQ_TRY(lnv_evaluate_corrected(s.get(), s->n_corr_initial));
    ctx->live_lnv.push_back(s.get());
    *out = s.release();
    return CQ_OK;
}

extern "C" cq_status cq_lnv_create(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                   const double *H, const cq_pattern *pL, double *L,
                                   double n_electrons, cq_precision prec, cq_lnv **out)
{
    if (!ctx || !pS) return CQ_ERR_INVALID;
    if (pS->n_cells() != 1)
        return cq_fail(ctx, CQ_ERR_INVALID, "lnv_create: batch patterns need cq_lnv_create_cells");
    return cq_lnv_create_cells(ctx, pS, S, H, pL, L, &n_electrons, prec, out);
}

extern "C" cq_status cq_lnv_step(cq_lnv *s, cq_lnv_report *rep)
{
    if (!s || !s->ctx) return CQ_ERR_INVALID;
    cq_ctx *ctx = s->ctx;
    const int nc = s->nc;
    const int64_t n = s->pL->n_values;
    const cq_pattern *pL = s->pL;
    double *G = s->G.as<double>(), *D = s->D.as<double>(), *GN = s->GN.as<double>();
    double *GE = s->GE.as<double>();
    const std::vector<double> one(nc, 1.0), zero(nc, 0.0), neg1(nc, -1.0);
    s->flops = 0.0;
    s->products = 0;
    std::vector<double> mu, gn2;
    CQ_TRY(lnv_mu_g(s, mu, gn2));
    // direction source Zc: G itself, or with a preconditioner Zs = sym(mask_L(T G T)); Zq is
    // the previous step's (G_prev, or Z_prev)
    const double *Zc = G, *Zq = s->Gp.as<double>();
    if (s->precond) {
        double *TG = s->TG.as<double>(), *Zr = s->Zr.as<double>(), *Zs = s->Zs.as<double>();
        const double *T = s->T.as<double>();
        CQ_TRY(bsmm(ctx, 1.0, s->pT, T, pL, G, 0.0, s->pTL, TG, s->prec, &s->flops));
        CQ_TRY(bsmm(ctx, 1.0, s->pTL, TG, s->pT, T, 0.0, pL, Zr, s->prec, &s->flops));
        s->products += 2;
        CQ_TRY(copy_vals(ctx, Zs, Zr, n));
        CQ_TRY(cq_gather(ctx, pL, Zr, pL, Zs, 1, 0.5, 0.5));  // Zs = (Zr + Zr^T) / 2
        Zc = Zs;
        Zq = s->Zp.as<double>();
    }
    std::vector<bool> restart(nc, !s->have_prev);
    if (!s->have_prev) {
        CQ_TRY(axpby_c(ctx, pL, neg1, Zc, zero, D));
    } else {
        // beta = max(0, <G, Z - Z_prev> / <G_prev, Z_prev>) (Z = G without a preconditioner),
        // D = -Z + beta D_prev
        CQ_TRY(copy_vals(ctx, D, Zc, n));
        CQ_TRY(axpby_c(ctx, pL, neg1, Zq, one, D));
        CQ_TRY(dot_q(ctx, pL, G, D, 0));
        CQ_TRY(dot_q(ctx, pL, s->Gp.as<double>(), Zq, 1));
        std::vector<std::vector<double>> d;
        CQ_TRY(fetch_q(ctx, nc, 2, d));
        std::vector<double> beta(nc);
        for (int c = 0; c < nc; ++c) beta[c] = std::fmax(0.0, d[0][c] / d[1][c]);
        CQ_TRY(copy_vals(ctx, D, s->Dp.as<double>(), n));
        CQ_TRY(axpby_c(ctx, pL, neg1, Zc, beta, D));
    }
    std::vector<double> dg;
    CQ_TRY(dots(s, D, GN, dg));
    std::vector<double> proj(nc);
    for (int c = 0; c < nc; ++c) proj[c] = -(dg[c] / gn2[c]);
    CQ_TRY(axpby_c(ctx, pL, proj, GN, one, D));
    std::vector<double> gd;
    CQ_TRY(dots(s, G, D, gd));
    bool any_restart = false;
    std::vector<double> ra(nc, 0.0), rb(nc, 1.0);
    for (int c = 0; c < nc; ++c)
        if (gd[c] >= 0.0) {
            restart[c] = true;
            any_restart = true;
            ra[c] = -1.0;
            rb[c] = 0.0;
        }
    if (any_restart) CQ_TRY(axpby_c(ctx, pL, ra, Zc, rb, D));
    std::vector<double> a1(nc), a2(nc);
    if (!s->have_alpha) {
        std::vector<double> gg;
        CQ_TRY(dots(s, Zc, Zc, gg));
        for (int c = 0; c < nc; ++c)
            a1[c] = 0.1 * std::sqrt((double)pL->seg_scalars[c]) / std::sqrt(gg[c]);
    } else {
        a1 = s->alpha_prev;
    }
    for (int c = 0; c < nc; ++c) a2[c] = 2.0 * a1[c];
    const std::vector<double> E0 = s->E, N0 = s->N;
    CQ_TRY(dot_q(ctx, pL, GE, D, 0));
    CQ_TRY(dot_q(ctx, pL, GN, D, 1));
    std::vector<std::vector<double>> g2;
    CQ_TRY(fetch_q(ctx, nc, 2, g2));
    const std::vector<double> &gE = g2[0], &gNd = g2[1];
    std::vector<double> E1, N1, E2, N2;
    double *Lt = s->Lt.as<double>();
    CQ_TRY(copy_vals(ctx, Lt, s->L, n));
    CQ_TRY(axpby_c(ctx, pL, a1, D, one, Lt));
    CQ_TRY(lnv_energy_number(s, Lt, E1, N1));
    CQ_TRY(copy_vals(ctx, Lt, s->L, n));
    CQ_TRY(axpby_c(ctx, pL, a2, D, one, Lt));
    CQ_TRY(lnv_energy_number(s, Lt, E2, N2));
    std::vector<double> alpha(nc);
    std::vector<bool> ok(nc);
    for (int c = 0; c < nc; ++c) {
        double e2, e3, n2, n3;
        cubic_coeffs(E0[c], gE[c], a1[c], E1[c], a2[c], E2[c], &e2, &e3);
        cubic_coeffs(N0[c], gNd[c], a1[c], N1[c], a2[c], N2[c], &n2, &n3);
        double a = 0.0;
        ok[c] = cubic_min(gE[c] - mu[c] * gNd[c], e2 - mu[c] * n2, e3 - mu[c] * n3, &a);
        alpha[c] = ok[c] ? a : 2.0 * a2[c];
    }
    // Without a minimiser the cubic falls without bound along D (the functional runs away
    // from idempotency): step 2*alpha_2, but at most until the RMS change of L reaches 0.01
    // per stored value.
    if (std::find(ok.begin(), ok.end(), false) != ok.end()) {
        std::vector<double> dd;
        CQ_TRY(dots(s, D, D, dd));
        for (int c = 0; c < nc; ++c)
            if (!ok[c] && dd[c] > 0.0)
                alpha[c] = std::fmin(alpha[c],
                                     0.01 * std::sqrt((double)pL->seg_scalars[c] / dd[c]));
    }
    CQ_TRY(axpby_c(ctx, pL, alpha, D, one, s->L));
    std::vector<int> ncorr;
    CQ_TRY(lnv_evaluate_corrected(s, ncorr));
    std::swap(s->G.ptr, s->Gp.ptr);  // G_prev <- G
    std::swap(s->D.ptr, s->Dp.ptr);  // D_prev <- D
    if (s->precond) std::swap(s->Zs.ptr, s->Zp.ptr);  // Z_prev <- Z
    s->have_prev = true;
    s->have_alpha = true;
    s->alpha_prev = alpha;
    if (rep) {
        CQ_TRY(lnv_report(s, rep));
        for (int c = 0; c < nc; ++c) {
            rep[c].alpha = alpha[c];
            rep[c].restart = restart[c] ? 1 : 0;
            rep[c].fallback = ok[c] ? 0 : 1;
            rep[c].n_corr = ncorr[c];
            rep[c].n_products = s->products;
            rep[c].flops = s->flops;
        }
    }
    return CQ_OK;
}

extern "C" cq_status cq_lnv_set_precision(cq_lnv *s, cq_precision prec)
{
    if (!s || !s->ctx) return CQ_ERR_INVALID;
    if (prec != CQ_FP64 && prec != CQ_SPLIT_BF16X3 && prec != CQ_FP64_EMU)
        return cq_fail(s->ctx, CQ_ERR_INVALID, "lnv_set_precision: unknown precision");
    s->prec = prec;
    s->have_prev = false;
    s->have_alpha = false;
    return lnv_evaluate_corrected(s, s->n_corr_initial);
}

extern "C" cq_status cq_lnv_set_preconditioner(cq_lnv *s, const cq_pattern *pT, const double *T)
{
    if (!s || !s->ctx) return CQ_ERR_INVALID;
    cq_ctx *ctx = s->ctx;
    s->have_prev = false;
    s->have_alpha = false;
    s->precond = false;  // stays off unless every step below succeeds
    if (!pT || !T) return CQ_OK;
    if (s->nc != 1)
        return cq_fail(ctx, CQ_ERR_INVALID, "lnv_set_preconditioner: single cells only");
    CQ_TRY(same_ctx(ctx, pT, s->pL));
    CQ_TRY(cq_pattern_derived(ctx, s->pL, 1.0, pT, 1.0, s->pL, &s->pTL));
    const size_t bl = sizeof(double) * s->pL->n_values;
    CQ_TRY(cq_alloc(ctx, s->T, sizeof(double) * pT->n_values));
    CQ_TRY(cq_alloc(ctx, s->TG, sizeof(double) * s->pTL->n_values));
    for (DevBuf *b : {&s->Zr, &s->Zs, &s->Zp}) CQ_TRY(cq_alloc(ctx, *b, bl));
    CQ_TRY(copy_vals(ctx, s->T.as<double>(), T, pT->n_values));
    s->pT = pT;
    s->precond = true;
    return cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "lnv_set_preconditioner");
}

extern "C" cq_status cq_lnv_state(const cq_lnv *cs, cq_lnv_report *rep)
{
    if (!cs || !rep || !cs->ctx) return CQ_ERR_INVALID;
    // the report needs G scratch: use Lt (not part of the state between steps)
    cq_lnv *s = const_cast<cq_lnv *>(cs);
    cq_ctx *ctx = s->ctx;
    const int nc = s->nc;
    CQ_TRY(dot_q(ctx, s->pL, s->GE.as<double>(), s->GN.as<double>(), 0));
    CQ_TRY(dot_q(ctx, s->pL, s->GN.as<double>(), s->GN.as<double>(), 1));
    std::vector<std::vector<double>> d;
    CQ_TRY(fetch_q(ctx, nc, 2, d));
    std::vector<double> neg(nc), one(nc, 1.0);
    for (int c = 0; c < nc; ++c) neg[c] = -(d[0][c] / d[1][c]);
    double *T = s->Lt.as<double>();
    CQ_TRY(copy_vals(ctx, T, s->GE.as<double>(), s->pL->n_values));
    CQ_TRY(axpby_c(ctx, s->pL, neg, s->GN.as<double>(), one, T));
    std::vector<double> gg;
    CQ_TRY(dots(s, T, T, gg));
    for (int c = 0; c < nc; ++c) {
        rep[c] = cq_lnv_report();
        rep[c].energy = s->E[c];
        rep[c].n_elec = s->N[c];
        rep[c].mu = -neg[c];
        rep[c].gnorm = std::sqrt(gg[c] / (double)s->pL->seg_scalars[c]);
        rep[c].n_corr = s->n_corr_initial[c];
    }
    return CQ_OK;
}

extern "C" cq_status cq_lnv_step_flops(cq_lnv *s, double *flops_host)
{
    if (!s || !flops_host || !s->ctx) return CQ_ERR_INVALID;
    TaskList *a, *b, *c;
    CQ_TRY(cq_get_tasks(s->ctx, s->pL, s->pS, s->pX, &a));
    CQ_TRY(cq_get_tasks(s->ctx, s->pS, s->pX, s->pU, &b));
    CQ_TRY(cq_get_tasks(s->ctx, s->pU, s->pX, s->pL, &c));
    // two trial points (X, Y, U, R1, R3) + one evaluation without corrections (7 products)
    *flops_host = 2.0 * (2 * a->flops + b->flops + 2 * c->flops) +
                  (2 * a->flops + 2 * b->flops + 3 * c->flops);
    if (s->precond) {  // T G on P_(T+L), then (T G) T on P_L
        TaskList *d, *e;
        CQ_TRY(cq_get_tasks(s->ctx, s->pT, s->pL, s->pTL, &d));
        CQ_TRY(cq_get_tasks(s->ctx, s->pTL, s->pT, s->pL, &e));
        *flops_host += d->flops + e->flops;
    }
    return CQ_OK;
}

extern "C" int32_t cq_lnv_cells(const cq_lnv *s) { return s ? s->nc : 0; }

void cq_lnv_detach(cq_lnv *s)
{
    s->ctx = nullptr;
    for (DevBuf *b : {&s->X, &s->Y, &s->U, &s->Z, &s->R1, &s->R2, &s->R3, &s->GE, &s->GN,
                      &s->G, &s->Gp, &s->D, &s->Dp, &s->Lt, &s->T, &s->TG, &s->Zr, &s->Zs,
                      &s->Zp})
        b->ctx = nullptr;
}

extern "C" void cq_lnv_destroy(cq_lnv *s)
{
    if (!s) return;
    if (s->ctx) {
        cudaStreamSynchronize(s->ctx->stream);
        auto &v = s->ctx->live_lnv;
        for (size_t e = 0; e < v.size(); ++e)
            if (v[e] == s) {
                v.erase(v.begin() + e);
                break;
            }
    }
    delete s;
}
