// Host drivers: Hotelling inversion, Palser-Manolopoulos start, McWeeny purification and the
// Li-Nunes-Vanderbilt minimisation.  All matrix work runs in the library's kernels; the
// host only does scalar arithmetic between phases (chemical potential, CG coefficients, the
// cubic line search) on FP64 scalars read back from device reductions.
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
    return cq_bsmm_split(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
}

#define CQ_TRY(x)                          \
    do {                                   \
        cq_status _st = (x);               \
        if (_st != CQ_OK) return _st;      \
    } while (0)

}  // namespace

// ---------------------------------------------------------------- Hotelling

extern "C" cq_status cq_hotelling_init(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                       const cq_pattern *pT, double *T)
{
    if (!ctx || !S || !T) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    CQ_TRY(cq_row_bounds_dev(ctx, pS, S, 0));
    double b[3];
    CQ_TRY(cq_fetch(ctx, 0, 3, b));
    if (!(b[2] > 0.0)) return cq_fail(ctx, CQ_ERR_NUMERIC, "hotelling_init: S has a zero row");
    return cq_set_identity(ctx, pT, T, 1.0 / b[2]);
}

extern "C" cq_status cq_hotelling_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                       const cq_pattern *pT, double *T, double *resid_host)
{
    if (!ctx || !S || !T) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    cq_pattern *pV = nullptr;
    CQ_TRY(cq_pattern_derived(ctx, pS, pS->range + pT->range, &pV));
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

// ---------------------------------------------------------------- PM start, McWeeny

extern "C" cq_status cq_pm_guess(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                 const double *H, const cq_pattern *pT, const double *T,
                                 const cq_pattern *pL, double *L, double n_occ)
{
    if (!ctx || !S || !H || !T || !L) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pT));
    CQ_TRY(same_ctx(ctx, pS, pL));
    const double n_orb = (double)pS->geo->n_orb;
    if (!(n_occ > 0.0 && n_occ < n_orb))
        return cq_fail(ctx, CQ_ERR_INVALID, "pm_guess: n_occ outside (0, N)");
    cq_pattern *pX = nullptr;
    CQ_TRY(cq_pattern_derived(ctx, pS, pT->range + pS->range, &pX));
    void *th;
    CQ_TRY(cq_scratch(ctx, "pm_TH", sizeof(double) * pX->n_values, &th));
    double *TH = (double *)th;
    CQ_TRY(bsmm(ctx, 1.0, pT, T, pS, H, 0.0, pX, TH, CQ_FP64));
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

extern "C" cq_status cq_mcweeny_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                     const cq_pattern *pL, double *L)
{
    if (!ctx || !S || !L) return CQ_ERR_INVALID;
    CQ_TRY(same_ctx(ctx, pS, pL));
    cq_pattern *pX, *pU, *p2L;
    CQ_TRY(cq_pattern_derived(ctx, pS, pL->range + pS->range, &pX));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0 * pS->range + pL->range, &pU));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0 * pL->range, &p2L));
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
    return cq_check_cuda(ctx, cudaMemcpyAsync(L, O, sizeof(double) * pL->n_values,
                                              cudaMemcpyDeviceToDevice, ctx->stream),
                         "mcweeny copy");
}

// ---------------------------------------------------------------- LNV

struct cq_lnv {
    cq_ctx *ctx = nullptr;
    const cq_pattern *pS = nullptr, *pL = nullptr;
    cq_pattern *pX = nullptr, *pU = nullptr;
    const double *S = nullptr, *H = nullptr;
    double *L = nullptr;
    double ne = 0.0;
    cq_precision prec = CQ_FP64;
    DevBuf X, Y, U, Z, R1, R2, R3, GE, GN, G, Gp, D, Dp, Lt;
    double E = 0.0, N = 0.0;
    bool have_prev = false, have_alpha = false;
    double alpha_prev = 0.0;
    double n_tol = 1e-10;
    double n_tol_split = 1e-9;
    int max_corr = 5;
    double flops = 0.0;
    int products = 0;
    int n_corr_initial = 0;
};

namespace {

// E and N at Lsrc from the five products a trial point needs (X, Y, U, R1, R3).
cq_status lnv_energy_number(cq_lnv *s, const double *Lsrc, double *E, double *N)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *Y = s->Y.as<double>(), *U = s->U.as<double>();
    double *R1 = s->R1.as<double>(), *R3 = s->R3.as<double>();
    CQ_TRY(bsmm(ctx, 1.0, s->pL, Lsrc, s->pS, s->S, 0.0, s->pX, X, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pL, Lsrc, s->pS, s->H, 0.0, s->pX, Y, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, X, 0.0, s->pU, U, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, Y, 0.0, s->pL, R1, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, X, 0.0, s->pL, R3, s->prec, &s->flops));
    s->products += 5;
    CQ_TRY(cq_trace_dev(ctx, s->pX, X, s->pX, Y, 0));
    CQ_TRY(cq_trace_dev(ctx, s->pL, Lsrc, s->pL, R1, 1));
    CQ_TRY(cq_trace_dev(ctx, s->pX, X, s->pX, X, 2));
    CQ_TRY(cq_trace_dev(ctx, s->pL, Lsrc, s->pL, R3, 3));
    double t[4];
    CQ_TRY(cq_fetch(ctx, 0, 4, t));
    *E = 2.0 * (3.0 * t[0] - 2.0 * t[1]);
    *N = 2.0 * (3.0 * t[2] - 2.0 * t[3]);
    return CQ_OK;
}

// Electron-number half of an evaluation at s->L: X = LS, U = SX, R3 = UX, N and G_N.
// (The products and values are those of a full evaluation; E and G_E follow in
// lnv_eval_rest at the same L.)
cq_status lnv_eval_n(cq_lnv *s)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *U = s->U.as<double>(), *R3 = s->R3.as<double>();
    CQ_TRY(bsmm(ctx, 1.0, s->pL, s->L, s->pS, s->S, 0.0, s->pX, X, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, X, 0.0, s->pU, U, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, X, 0.0, s->pL, R3, s->prec, &s->flops));
    s->products += 3;
    CQ_TRY(cq_trace_dev(ctx, s->pX, X, s->pX, X, 2));
    CQ_TRY(cq_trace_dev(ctx, s->pL, s->L, s->pL, R3, 3));
    CQ_TRY(cq_lnv_gradient_n(ctx, s->pL, s->pU, U, R3, s->GN.as<double>()));
    double t[2];
    CQ_TRY(cq_fetch(ctx, 2, 2, t));
    s->N = 2.0 * (3.0 * t[0] - 2.0 * t[1]);
    return CQ_OK;
}

// Energy half at the L of the last lnv_eval_n (X, U still current): Y = LH, R1 = UY,
// Z = SY, R2 = ZX, E and G_E.
cq_status lnv_eval_rest(cq_lnv *s)
{
    cq_ctx *ctx = s->ctx;
    double *X = s->X.as<double>(), *Y = s->Y.as<double>(), *U = s->U.as<double>();
    double *Z = s->Z.as<double>(), *R1 = s->R1.as<double>(), *R2 = s->R2.as<double>();
    CQ_TRY(bsmm(ctx, 1.0, s->pL, s->L, s->pS, s->H, 0.0, s->pX, Y, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pU, U, s->pX, Y, 0.0, s->pL, R1, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pS, s->S, s->pX, Y, 0.0, s->pU, Z, s->prec, &s->flops));
    CQ_TRY(bsmm(ctx, 1.0, s->pU, Z, s->pX, X, 0.0, s->pL, R2, s->prec, &s->flops));
    s->products += 4;
    CQ_TRY(cq_trace_dev(ctx, s->pX, X, s->pX, Y, 0));
    CQ_TRY(cq_trace_dev(ctx, s->pL, s->L, s->pL, R1, 1));
    CQ_TRY(cq_lnv_gradient_e(ctx, s->pL, s->pU, Z, R1, R2, s->GE.as<double>()));
    double t[2];
    CQ_TRY(cq_fetch(ctx, 0, 2, t));
    s->E = 2.0 * (3.0 * t[0] - 2.0 * t[1]);
    return CQ_OK;
}

cq_status dot_l(cq_lnv *s, const double *a, const double *b, double *out)
{
    CQ_TRY(cq_dot_dev(s->ctx, s->pL, a, b, 0));
    return cq_fetch(s->ctx, 0, 1, out);
}

// Evaluate at s->L with the electron-number corrections in between: N and G_N first, then
// L += ((N_e - N)/<G_N,G_N>) G_N (at most max_corr times) while |N - N_e| > n_tol N_e, each
// followed by N and G_N at the corrected L, and finally E and G_E at the last L.  The
// iterates and decisions are those of "full evaluation, then correct and re-evaluate";
// only the E half of the intermediate evaluations (never used) is skipped.
cq_status lnv_evaluate_corrected(cq_lnv *s, int *count)
{
    CQ_TRY(lnv_eval_n(s));
    int k = 0;
    // split-BF16 products resolve N to ~1e-10 relative, so their corrections stop at 1e-9
    const double tol = s->prec == CQ_SPLIT_BF16X3 ? s->n_tol_split : s->n_tol;
    while (std::fabs(s->N - s->ne) > tol * s->ne && k < s->max_corr) {
        double gn2;
        CQ_TRY(dot_l(s, s->GN.as<double>(), s->GN.as<double>(), &gn2));
        CQ_TRY(cq_axpby(s->ctx, s->pL->n_values, (s->ne - s->N) / gn2, s->GN.as<double>(), 1.0,
                        s->L));
        CQ_TRY(lnv_eval_n(s));
        ++k;
    }
    *count = k;
    return lnv_eval_rest(s);
}

// mu = <G_E,G_N>/<G_N,G_N> and G = G_E - mu G_N into s->G; returns <G_N,G_N>.
cq_status lnv_mu_g(cq_lnv *s, double *mu, double *gn2)
{
    cq_ctx *ctx = s->ctx;
    CQ_TRY(cq_dot_dev(ctx, s->pL, s->GE.as<double>(), s->GN.as<double>(), 0));
    CQ_TRY(cq_dot_dev(ctx, s->pL, s->GN.as<double>(), s->GN.as<double>(), 1));
    double d[2];
    CQ_TRY(cq_fetch(ctx, 0, 2, d));
    *mu = d[0] / d[1];
    *gn2 = d[1];
    CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(s->G.ptr, s->GE.ptr, sizeof(double) * s->pL->n_values,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    return cq_axpby(ctx, s->pL->n_values, -*mu, s->GN.as<double>(), 1.0, s->G.as<double>());
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
    double mu, gn2, gg;
    CQ_TRY(lnv_mu_g(s, &mu, &gn2));
    CQ_TRY(dot_l(s, s->G.as<double>(), s->G.as<double>(), &gg));
    rep->energy = s->E;
    rep->n_elec = s->N;
    rep->mu = mu;
    rep->gnorm = std::sqrt(gg / (double)s->pL->n_scalars);
    return CQ_OK;
}

}  // namespace

extern "C" cq_status cq_lnv_create(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                   const double *H, const cq_pattern *pL, double *L,
                                   double n_electrons, cq_precision prec, cq_lnv **out)
{
    if (!ctx || !out || !S || !H || !L) return CQ_ERR_INVALID;
    *out = nullptr;
    CQ_TRY(same_ctx(ctx, pS, pL));
    if (!(n_electrons > 0.0 && n_electrons < 2.0 * (double)pS->geo->n_orb))
        return cq_fail(ctx, CQ_ERR_INVALID, "lnv_create: electron count outside (0, 2N)");
    if (prec != CQ_FP64 && prec != CQ_SPLIT_BF16X3)
        return cq_fail(ctx, CQ_ERR_INVALID, "lnv_create: unknown precision");
    std::unique_ptr<cq_lnv> s(new cq_lnv());
    s->ctx = ctx;
    s->pS = pS;
    s->pL = pL;
    s->S = S;
    s->H = H;
    s->L = L;
    s->ne = n_electrons;
    s->prec = prec;
    CQ_TRY(cq_pattern_derived(ctx, pS, pL->range + pS->range, &s->pX));
    CQ_TRY(cq_pattern_derived(ctx, pS, 2.0 * pS->range + pL->range, &s->pU));
    const size_t bx = sizeof(double) * s->pX->n_values, bu = sizeof(double) * s->pU->n_values;
    const size_t bl = sizeof(double) * pL->n_values;
    CQ_TRY(cq_alloc(ctx, s->X, bx));
    CQ_TRY(cq_alloc(ctx, s->Y, bx));
    CQ_TRY(cq_alloc(ctx, s->U, bu));
    CQ_TRY(cq_alloc(ctx, s->Z, bu));
    for (DevBuf *b : {&s->R1, &s->R2, &s->R3, &s->GE, &s->GN, &s->G, &s->Gp, &s->D, &s->Dp, &s->Lt})
        CQ_TRY(cq_alloc(ctx, *b, bl));
    CQ_TRY(lnv_evaluate_corrected(s.get(), &s->n_corr_initial));
    ctx->live_lnv.push_back(s.get());
    *out = s.release();
    return CQ_OK;
}

extern "C" cq_status cq_lnv_step(cq_lnv *s, cq_lnv_report *rep)
{
    if (!s || !s->ctx) return CQ_ERR_INVALID;
    cq_ctx *ctx = s->ctx;
    const int64_t n = s->pL->n_values;
    double *G = s->G.as<double>(), *D = s->D.as<double>(), *GN = s->GN.as<double>();
    double *GE = s->GE.as<double>();
    s->flops = 0.0;
    s->products = 0;
    double mu, gn2;
    CQ_TRY(lnv_mu_g(s, &mu, &gn2));
    bool restart = !s->have_prev;
    if (restart) {
        CQ_TRY(cq_axpby(ctx, n, -1.0, G, 0.0, D));
    } else {
        // beta = max(0, <G, G - G_prev> / <G_prev, G_prev>), D = -G + beta D_prev
        CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(D, G, sizeof(double) * n,
                                                  cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
        CQ_TRY(cq_axpby(ctx, n, -1.0, s->Gp.as<double>(), 1.0, D));
        CQ_TRY(cq_dot_dev(ctx, s->pL, G, D, 0));
        CQ_TRY(cq_dot_dev(ctx, s->pL, s->Gp.as<double>(), s->Gp.as<double>(), 1));
        double d[2];
        CQ_TRY(cq_fetch(ctx, 0, 2, d));
        const double beta = std::fmax(0.0, d[0] / d[1]);
        CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(D, s->Dp.ptr, sizeof(double) * n,
                                                  cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
        CQ_TRY(cq_axpby(ctx, n, -1.0, G, beta, D));
    }
    double dg;
    CQ_TRY(dot_l(s, D, GN, &dg));
    CQ_TRY(cq_axpby(ctx, n, -(dg / gn2), GN, 1.0, D));
    double gd;
    CQ_TRY(dot_l(s, G, D, &gd));
    if (gd >= 0.0) {
        CQ_TRY(cq_axpby(ctx, n, -1.0, G, 0.0, D));
        restart = true;
    }
    double a1;
    if (!s->have_alpha) {
        double gg;
        CQ_TRY(dot_l(s, G, G, &gg));
        a1 = 0.1 * std::sqrt((double)s->pL->n_scalars) / std::sqrt(gg);
    } else {
        a1 = s->alpha_prev;
    }
    const double a2 = 2.0 * a1;
    const double E0 = s->E, N0 = s->N;
    CQ_TRY(cq_dot_dev(ctx, s->pL, GE, D, 0));
    CQ_TRY(cq_dot_dev(ctx, s->pL, GN, D, 1));
    double g2[2];
    CQ_TRY(cq_fetch(ctx, 0, 2, g2));
    const double gE = g2[0], gNd = g2[1];
    double E1, N1, E2, N2;
    double *Lt = s->Lt.as<double>();
    CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(Lt, s->L, sizeof(double) * n,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    CQ_TRY(cq_axpby(ctx, n, a1, D, 1.0, Lt));
    CQ_TRY(lnv_energy_number(s, Lt, &E1, &N1));
    CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(Lt, s->L, sizeof(double) * n,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    CQ_TRY(cq_axpby(ctx, n, a2, D, 1.0, Lt));
    CQ_TRY(lnv_energy_number(s, Lt, &E2, &N2));
    double e2, e3, n2, n3;
    cubic_coeffs(E0, gE, a1, E1, a2, E2, &e2, &e3);
    cubic_coeffs(N0, gNd, a1, N1, a2, N2, &n2, &n3);
    double alpha = 0.0;
    const bool ok = cubic_min(gE - mu * gNd, e2 - mu * n2, e3 - mu * n3, &alpha);
    if (!ok) alpha = 2.0 * a2;
    CQ_TRY(cq_axpby(ctx, n, alpha, D, 1.0, s->L));
    int ncorr = 0;
    CQ_TRY(lnv_evaluate_corrected(s, &ncorr));
    std::swap(s->G.ptr, s->Gp.ptr);  // G_prev <- G
    std::swap(s->D.ptr, s->Dp.ptr);  // D_prev <- D
    s->have_prev = true;
    s->have_alpha = true;
    s->alpha_prev = alpha;
    if (rep) {
        CQ_TRY(lnv_report(s, rep));
        rep->alpha = alpha;
        rep->restart = restart ? 1 : 0;
        rep->fallback = ok ? 0 : 1;
        rep->n_corr = ncorr;
        rep->n_products = s->products;
        rep->flops = s->flops;
    }
    return CQ_OK;
}

extern "C" cq_status cq_lnv_set_precision(cq_lnv *s, cq_precision prec)
{
    if (!s || !s->ctx) return CQ_ERR_INVALID;
    if (prec != CQ_FP64 && prec != CQ_SPLIT_BF16X3)
        return cq_fail(s->ctx, CQ_ERR_INVALID, "lnv_set_precision: unknown precision");
    s->prec = prec;
    s->have_prev = false;
    s->have_alpha = false;
    return lnv_evaluate_corrected(s, &s->n_corr_initial);
}

extern "C" cq_status cq_lnv_state(const cq_lnv *s, cq_lnv_report *rep)
{
    if (!s || !rep || !s->ctx) return CQ_ERR_INVALID;
    // the report needs G scratch: use Lt (not part of the state between steps)
    cq_lnv *m = const_cast<cq_lnv *>(s);
    cq_ctx *ctx = m->ctx;
    double d[2];
    CQ_TRY(cq_dot_dev(ctx, m->pL, m->GE.as<double>(), m->GN.as<double>(), 0));
    CQ_TRY(cq_dot_dev(ctx, m->pL, m->GN.as<double>(), m->GN.as<double>(), 1));
    CQ_TRY(cq_fetch(ctx, 0, 2, d));
    const double mu = d[0] / d[1];
    double *T = m->Lt.as<double>();
    CQ_TRY(cq_check_cuda(ctx, cudaMemcpyAsync(T, m->GE.ptr, sizeof(double) * m->pL->n_values,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "copy"));
    CQ_TRY(cq_axpby(ctx, m->pL->n_values, -mu, m->GN.as<double>(), 1.0, T));
    double gg;
    CQ_TRY(dot_l(m, T, T, &gg));
    *rep = cq_lnv_report();
    rep->energy = m->E;
    rep->n_elec = m->N;
    rep->mu = mu;
    rep->gnorm = std::sqrt(gg / (double)m->pL->n_scalars);
    rep->n_corr = m->n_corr_initial;
    return CQ_OK;
}

extern "C" cq_status cq_lnv_step_flops(cq_lnv *s, double *flops_host)
{
    if (!s || !flops_host || !s->ctx) return CQ_ERR_INVALID;
    TaskList *a, *b, *c;
    CQ_TRY(cq_get_tasks(s->ctx, s->pL, s->pS, s->pX, &a));
    CQ_TRY(cq_get_tasks(s->ctx, s->pS, s->pX, s->pU, &b));
    CQ_TRY(cq_get_tasks(s->ctx, s->pU, s->pX, s->pL, &c));
    // full evaluation (X, Y, U, Z, R1, R2, R3) + two trial points (X, Y, U, R1, R3)
    *flops_host = (2 * a->flops + 2 * b->flops + 3 * c->flops) +
                  2.0 * (2 * a->flops + b->flops + 2 * c->flops);
    return CQ_OK;
}

void cq_lnv_detach(cq_lnv *s)
{
    s->ctx = nullptr;
    for (DevBuf *b : {&s->X, &s->Y, &s->U, &s->Z, &s->R1, &s->R2, &s->R3, &s->GE, &s->GN,
                      &s->G, &s->Gp, &s->D, &s->Dp, &s->Lt})
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
