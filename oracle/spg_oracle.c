/*
 * FP64 CPU oracle for the reweighted smoothing-proximal-gradient solve of the
 * regularized real-space refinement objective (Luo, arXiv 1905.13408, Sec. 2.1
 * and Sec. 2.5).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the package's smoke check and the
 * benchmark's CPU-baseline leg are its only callers; the CUDA library never
 * links, loads or calls it, and it shares no code with the CUDA library.
 *
 * Everything is double precision, plain loops over a [nz][ny][nx] volume
 * (x fastest), no tiling and no fusion beyond what each definition states.
 * OpenMP only splits loops over z-planes; every reduction is summed per plane
 * and then over planes in a fixed order, so results do not depend on the
 * thread count.
 *
 * Objective minimised in round r (the negative of the paper's maximisation,
 * Eq. 11 and the matrix form Eq. 31 with the real-space diagonal data term of
 * Eq. 28):
 *
 *   F(x) = 1/2 sum_v w_v (x_v - b_v)^2
 *        + lambda_l1 sum_v om1_v |x_v|
 *        + lambda_tv sum_v omtv_v h_mu((Dx)_v)
 *
 *   (Dx)_{v,a} = x_v - x_{v - e_a} if v_a >= 1, else 0        (Eq. 12)
 *   h_mu(z)    = max_{|u|<=1} <u,z> - mu/2 |u|^2               (Eq. 14)
 *              = |z|^2/(2 mu) if |z| <= mu, |z| - mu/2 otherwise
 *   grad h_mu(z) = z / max(mu, |z|)                            (Eq. 16)
 *   (D^T u)_v  = sum_a [v_a>=1] u_a[v] - [v_a+1<=n_a-1] u_a[v+e_a]   (Eq. 17)
 *   om1_v  = eps    / (|x^r_v| + eps)                          (Eq. 11 x eps, Sec. 2.5)
 *   omtv_v = eps_tv / (|(Dx^r)_v| + eps_tv)
 *
 * One step (Eq. 20 and Eq. 21, with FISTA extrapolation; beta = 0 gives the
 * paper's plain proximal-gradient update):
 *
 *   y      = x_k + beta_k (x_k - x_{k-1})
 *   z      = y - tau (w (y - b) + lambda_tv D^T(omtv grad h_mu(D y)))
 *   x_{k+1} = soft(z, tau lambda_l1 om1)
 *
 * with tau = 1/L, L = max w + 12 lambda_tv max(omtv) / mu.
 *
 * Alternative readings of the paper are flags of orc_params (forward
 * differences, periodic boundary, TV weight after the divergence); the
 * per-voxel sampled step and the adjoint implement the adopted readings only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double lambda_l1, lambda_tv, mu, eps, eps_tv;
    int momentum; /* 0: FISTA extrapolation, 1: plain proximal gradient (beta = 0) */
    int restart;  /* 1: restart the extrapolation whenever <y_k - x_{k+1}, x_{k+1} - x_k> > 0 */
    double gamma;          /* weight of the implicit-gradient term gamma |x - anchor|^2 (Eq. 22) */
    const double *anchor;  /* the previous maximisation step's solution; used when gamma > 0 */
    /* Alternative readings of the paper (the adopted ones are all 0):
     * forward:  forward differences x_{v+e_a} - x_v instead of Eq. 12's backward ones;
     * periodic: differences wrap around the volume instead of vanishing at its edge;
     * post_div: the TV weight multiplies the divergence, omtv * D^T(grad h_mu(D x))
     *           (Eq. 20 as printed), instead of D^T(omtv grad h_mu(D x)). */
    int forward, periodic, post_div;
} orc_params;

#define NVOX(p) ((size_t)(p)->nx * (size_t)(p)->ny * (size_t)(p)->nz)
#define AT(p, x, y, z) ((((size_t)(z) * (size_t)(p)->ny) + (size_t)(y)) * (size_t)(p)->nx + (size_t)(x))

/* ---------- closed forms (Eq. 14, Eq. 16, Eq. 21) ---------- */

/* Weighted soft-threshold, Eq. 21: 0 if |z| < t, z - t sign(z) otherwise. */
double orc_soft(double z, double t)
{
    if (fabs(z) < t) return 0.0;
    return z > 0.0 ? z - t : z + t;
}

/* Nesterov-smoothed Euclidean norm of a 3-vector, Eq. 14 in closed form. */
double orc_huber(double z0, double z1, double z2, double mu)
{
    double s2 = z0 * z0 + z1 * z1 + z2 * z2;
    double s = sqrt(s2);
    if (s <= mu) return s2 / (2.0 * mu);
    return s - 0.5 * mu;
}

/* Gradient of the smoothed norm, Eq. 16: z / max(mu, |z|). */
void orc_huber_grad(double z0, double z1, double z2, double mu, double out[3])
{
    double s = sqrt(z0 * z0 + z1 * z1 + z2 * z2);
    double d = s > mu ? s : mu;
    out[0] = z0 / d;
    out[1] = z1 / d;
    out[2] = z2 / d;
}

/* ---------- linear operators (Eq. 12, Eq. 17) ---------- */

/* Coordinate c of axis a (extent na) shifted by d, wrapped modulo na. */
static int wrapc(int c, int d, int na) { return ((c + d) % na + na) % na; }

/* Whether the difference of axis a at coordinate c exists (it is 0 otherwise):
 * backward needs the voxel at c - 1, forward the voxel at c + 1; with the
 * periodic boundary every difference exists. */
static int has_diff(const orc_params *p, int c, int na)
{
    if (p->periodic) return 1;
    return p->forward ? c + 1 <= na - 1 : c >= 1;
}

static size_t at_axis(const orc_params *p, int xx, int y, int z, int a, int c)
{
    if (a == 0) return AT(p, c, y, z);
    if (a == 1) return AT(p, xx, c, z);
    return AT(p, xx, y, c);
}

/* g[a*n + v] = (Dx)_{v,a}, a = 0 (x), 1 (y), 2 (z). Adopted reading: backward
 * differences (Eq. 12), zero on the first plane of each axis (Neumann). */
void orc_grad(const orc_params *p, const double *x, double *g)
{
    const size_t n = NVOX(p);
    const int ext[3] = {p->nx, p->ny, p->nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int xx = 0; xx < p->nx; xx++) {
                const size_t v = AT(p, xx, y, z);
                const int co[3] = {xx, y, z};
                for (int a = 0; a < 3; a++) {
                    const int c = co[a], na = ext[a];
                    double d = 0.0;
                    if (has_diff(p, c, na)) {
                        if (p->forward)
                            d = x[at_axis(p, xx, y, z, a, wrapc(c, 1, na))] - x[v];
                        else
                            d = x[v] - x[at_axis(p, xx, y, z, a, wrapc(c, -1, na))];
                    }
                    g[(size_t)a * n + v] = d;
                }
            }
}

/* out = D^T u, the adjoint of orc_grad (Eq. 17 for the adopted reading): x_v
 * enters the difference at v with sign +1 (backward) or -1 (forward), and the
 * difference at its successor v + e_a (backward, sign -1) or predecessor
 * v - e_a (forward, sign +1) whenever that difference exists. */
void orc_div(const orc_params *p, const double *u, double *out)
{
    const size_t n = NVOX(p);
    const int ext[3] = {p->nx, p->ny, p->nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int xx = 0; xx < p->nx; xx++) {
                const size_t v = AT(p, xx, y, z);
                const int co[3] = {xx, y, z};
                double s = 0.0;
                for (int a = 0; a < 3; a++) {
                    const double *ua = u + (size_t)a * n;
                    const int c = co[a], na = ext[a];
                    if (!p->forward) {
                        if (has_diff(p, c, na)) s += ua[v];
                        if (p->periodic || c + 1 <= na - 1) s -= ua[at_axis(p, xx, y, z, a, wrapc(c, 1, na))];
                    } else {
                        if (has_diff(p, c, na)) s -= ua[v];
                        if (p->periodic || c >= 1) s += ua[at_axis(p, xx, y, z, a, wrapc(c, -1, na))];
                    }
                }
                out[v] = s;
            }
}

/* Gradient of the weighted smoothed TV term (without lambda_tv):
 * D^T(omtv * grad h_mu(D x)), Eq. 15-17 with the Eq. 11 weights inside
 * (with post_div: omtv * D^T(grad h_mu(D x)), which is not the gradient of
 * any objective unless omtv is constant). */
void orc_tv_grad(const orc_params *p, const double *x, const double *omtv, double *out)
{
    const size_t n = NVOX(p);
    double *g = (double *)malloc(3 * n * sizeof(double));
    orc_grad(p, x, g);
#pragma omp parallel for schedule(static)
    for (long long v = 0; v < (long long)n; v++) {
        double u[3];
        orc_huber_grad(g[v], g[n + v], g[2 * n + v], p->mu, u);
        double om = (omtv && !p->post_div) ? omtv[v] : 1.0;
        g[v] = om * u[0];
        g[n + v] = om * u[1];
        g[2 * n + v] = om * u[2];
    }
    orc_div(p, g, out);
    if (p->post_div && omtv) {
#pragma omp parallel for schedule(static)
        for (long long v = 0; v < (long long)n; v++) out[v] *= omtv[v];
    }
    free(g);
}

/* Gradient of the smooth part f = data + TV (+ the Eq. 22 term):
 * w (x - b) + lambda_tv D^T(...) + 2 gamma (x - anchor). */
void orc_grad_f(const orc_params *p, const double *x, const double *b, const double *w,
                const double *omtv, double *out)
{
    const size_t n = NVOX(p);
    orc_tv_grad(p, x, omtv, out);
#pragma omp parallel for schedule(static)
    for (long long v = 0; v < (long long)n; v++) {
        out[v] = w[v] * (x[v] - b[v]) + p->lambda_tv * out[v];
        if (p->gamma > 0.0) out[v] += 2.0 * p->gamma * (x[v] - p->anchor[v]);
    }
}

/* ---------- objective, weights, step size ---------- */

/* out = {data, l1, tv, total} of F at x (Eq. 31 form, Eq. 14 smoothed TV);
 * with gamma > 0 the data part includes gamma |x - anchor|^2 (Eq. 22). */
void orc_objective(const orc_params *p, const double *x, const double *b, const double *w,
                   const double *om1, const double *omtv, double out[4])
{
    const size_t n = NVOX(p);
    double *g = (double *)malloc(3 * n * sizeof(double));
    double *pd = (double *)calloc((size_t)p->nz, sizeof(double));
    double *pl = (double *)calloc((size_t)p->nz, sizeof(double));
    double *pt = (double *)calloc((size_t)p->nz, sizeof(double));
    orc_grad(p, x, g);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++) {
        double sd = 0.0, sl = 0.0, st = 0.0;
        for (int y = 0; y < p->ny; y++)
            for (int xx = 0; xx < p->nx; xx++) {
                size_t v = AT(p, xx, y, z);
                double r = x[v] - b[v];
                sd += 0.5 * w[v] * r * r;
                if (p->gamma > 0.0) sd += p->gamma * (x[v] - p->anchor[v]) * (x[v] - p->anchor[v]);
                sl += (om1 ? om1[v] : 1.0) * fabs(x[v]);
                st += (omtv ? omtv[v] : 1.0) * orc_huber(g[v], g[n + v], g[2 * n + v], p->mu);
            }
        pd[z] = sd;
        pl[z] = sl;
        pt[z] = st;
    }
    double sd = 0.0, sl = 0.0, st = 0.0;
    for (int z = 0; z < p->nz; z++) {
        sd += pd[z];
        sl += pl[z];
        st += pt[z];
    }
    out[0] = sd;
    out[1] = p->lambda_l1 * sl;
    out[2] = p->lambda_tv * st;
    out[3] = out[0] + out[1] + out[2];
    free(g);
    free(pd);
    free(pl);
    free(pt);
}

/* Re-weighting between rounds (Eq. 11 weights scaled by eps as in Sec. 2.5).
 * stats = {max omtv, count of nonzero x, sum om1, sum omtv}. */
void orc_reweight(const orc_params *p, const double *x, double *om1, double *omtv, double stats[4])
{
    const size_t n = NVOX(p);
    double *g = (double *)malloc(3 * n * sizeof(double));
    double *pm = (double *)calloc((size_t)p->nz, sizeof(double));
    double *pn = (double *)calloc((size_t)p->nz, sizeof(double));
    double *p1 = (double *)calloc((size_t)p->nz, sizeof(double));
    double *p2 = (double *)calloc((size_t)p->nz, sizeof(double));
    orc_grad(p, x, g);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++) {
        double m = 0.0, c = 0.0, s1 = 0.0, s2 = 0.0;
        for (int y = 0; y < p->ny; y++)
            for (int xx = 0; xx < p->nx; xx++) {
                size_t v = AT(p, xx, y, z);
                double gn = sqrt(g[v] * g[v] + g[n + v] * g[n + v] + g[2 * n + v] * g[2 * n + v]);
                om1[v] = p->eps / (fabs(x[v]) + p->eps);
                omtv[v] = p->eps_tv / (gn + p->eps_tv);
                if (omtv[v] > m) m = omtv[v];
                if (x[v] != 0.0) c += 1.0;
                s1 += om1[v];
                s2 += omtv[v];
            }
        pm[z] = m;
        pn[z] = c;
        p1[z] = s1;
        p2[z] = s2;
    }
    stats[0] = 0.0;
    stats[1] = 0.0;
    stats[2] = 0.0;
    stats[3] = 0.0;
    for (int z = 0; z < p->nz; z++) {
        if (pm[z] > stats[0]) stats[0] = pm[z];
        stats[1] += pn[z];
        stats[2] += p1[z];
        stats[3] += p2[z];
    }
    free(g);
    free(pm);
    free(pn);
    free(p1);
    free(p2);
}

/* Lipschitz bound of grad f: max w + |D|^2 lambda_tv max(omtv) / mu (+ 2 gamma), |D|^2 <= 12. */
double orc_lipschitz(const orc_params *p, const double *w, double max_omtv)
{
    const size_t n = NVOX(p);
    double m = 0.0;
    for (size_t v = 0; v < n; v++)
        if (w[v] > m) m = w[v];
    return m + 12.0 * p->lambda_tv * max_omtv / p->mu + 2.0 * (p->gamma > 0.0 ? p->gamma : 0.0);
}

/* FISTA extrapolation weights: t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
 * beta_k = (t_k - 1)/t_{k+1}; all zero for the plain proximal-gradient update. */
void orc_beta_table(int momentum, int iters, double *beta)
{
    double t = 1.0;
    for (int k = 0; k < iters; k++) {
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        beta[k] = momentum == 0 ? (t - 1.0) / tn : 0.0;
        t = tn;
    }
}

/* ---------- one step and the full schedule ---------- */

/* x_next = soft(y - tau grad f(y), tau lambda_l1 om1), y = x_k + beta (x_k - x_km1). */
void orc_step(const orc_params *p, const double *xk, const double *xkm1, double beta, double tau,
              const double *b, const double *w, const double *om1, const double *omtv, double *xnext)
{
    const size_t n = NVOX(p);
    double *y = (double *)malloc(n * sizeof(double));
    double *g = (double *)malloc(n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long long v = 0; v < (long long)n; v++) y[v] = xk[v] + beta * (xk[v] - xkm1[v]);
    orc_grad_f(p, y, b, w, omtv, g);
#pragma omp parallel for schedule(static)
    for (long long v = 0; v < (long long)n; v++)
        xnext[v] = orc_soft(y[v] - tau * g[v], tau * p->lambda_l1 * (om1 ? om1[v] : 1.0));
    free(y);
    free(g);
}

/* <y - x_next, x_next - x> with y = x + beta (x - xprev), summed per z-plane
 * and then over planes in order (the gradient restart test of O'Donoghue and
 * Candes, 2015: restart when the step moves against the extrapolation). */
static double restart_dot(const orc_params *p, const double *x, const double *xprev, const double *xnext,
                          double beta)
{
    double *pz = (double *)calloc((size_t)p->nz, sizeof(double));
    const size_t plane = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++) {
        double s = 0.0;
        for (size_t v = (size_t)z * plane; v < (size_t)(z + 1) * plane; v++) {
            double y = x[v] + beta * (x[v] - xprev[v]);
            s += (y - xnext[v]) * (xnext[v] - x[v]);
        }
        pz[z] = s;
    }
    double s = 0.0;
    for (int z = 0; z < p->nz; z++) s += pz[z];
    free(pz);
    return s;
}

/* Reweighted solve: `rounds` rounds of `iters` steps from the given x (in/out).
 * Round r re-weights from the current x, sets tau = 1/L and restarts the
 * momentum (x_{-1} = x_0, t = 1). With p->restart the extrapolation index
 * also returns to 0 after any step whose restart_dot is positive.
 * hist (optional): rounds*iters*4 doubles, F(x_k) before step k of round r.
 * rstats (optional): rounds*6 doubles = {max omtv, nnz, sum om1, sum omtv, L, tau}.
 * om1_out/omtv_out (optional): the weights of the last round. */
int orc_solve(const orc_params *p, const double *b, const double *w, int rounds, int iters,
              double *x, double *hist, double *rstats, double *om1_out, double *omtv_out)
{
    const size_t n = NVOX(p);
    double *om1 = (double *)malloc(n * sizeof(double));
    double *omtv = (double *)malloc(n * sizeof(double));
    double *xprev = (double *)malloc(n * sizeof(double));
    double *xnext = (double *)malloc(n * sizeof(double));
    double *beta = (double *)malloc((size_t)(iters > 0 ? iters : 1) * sizeof(double));
    if (!om1 || !omtv || !xprev || !xnext || !beta) return -1;
    orc_beta_table(p->momentum, iters, beta);
    for (int r = 0; r < rounds; r++) {
        double st[4];
        orc_reweight(p, x, om1, omtv, st);
        double L = orc_lipschitz(p, w, st[0]);
        double tau = 1.0 / L;
        if (rstats) {
            for (int i = 0; i < 4; i++) rstats[r * 6 + i] = st[i];
            rstats[r * 6 + 4] = L;
            rstats[r * 6 + 5] = tau;
        }
        memcpy(xprev, x, n * sizeof(double));
        int km = 0; /* index into the extrapolation table */
        for (int k = 0; k < iters; k++) {
            if (hist) orc_objective(p, x, b, w, om1, omtv, hist + ((size_t)r * iters + k) * 4);
            orc_step(p, x, xprev, beta[km], tau, b, w, om1, omtv, xnext);
            if (p->restart && restart_dot(p, x, xprev, xnext, beta[km]) > 0.0)
                km = 0;
            else
                km++;
            memcpy(xprev, x, n * sizeof(double));
            memcpy(x, xnext, n * sizeof(double));
        }
    }
    if (om1_out) memcpy(om1_out, om1, n * sizeof(double));
    if (omtv_out) memcpy(omtv_out, omtv, n * sizeof(double));
    free(om1);
    free(omtv);
    free(xprev);
    free(xnext);
    free(beta);
    return 0;
}

/* K steps of one round with fixed weights and step: x_K from x_0 (x_{-1} = x_0). */
void orc_unrolled(const orc_params *p, const double *b, const double *w, const double *om1,
                  const double *omtv, double tau, int iters, const double *x0, double *xK)
{
    const size_t n = NVOX(p);
    double *xc = (double *)malloc(n * sizeof(double));
    double *xp = (double *)malloc(n * sizeof(double));
    double *xn = (double *)malloc(n * sizeof(double));
    double *beta = (double *)malloc((size_t)(iters > 0 ? iters : 1) * sizeof(double));
    orc_beta_table(p->momentum, iters, beta);
    memcpy(xc, x0, n * sizeof(double));
    memcpy(xp, x0, n * sizeof(double));
    for (int k = 0; k < iters; k++) {
        orc_step(p, xc, xp, beta[k], tau, b, w, om1, omtv, xn);
        double *t = xp;
        xp = xc;
        xc = xn;
        xn = t;
    }
    memcpy(xK, xc, n * sizeof(double));
    free(xc);
    free(xp);
    free(xn);
    free(beta);
}

/* As orc_unrolled, and counts the voxel-steps where the soft-threshold
 * passes (|z| > t, or t = 0): two runs with equal counts crossed no kink of
 * Eq. 21 in different places unless changes cancel exactly. */
long long orc_unrolled_active(const orc_params *p, const double *b, const double *w, const double *om1,
                              const double *omtv, double tau, int iters, const double *x0, double *xK)
{
    const size_t n = NVOX(p);
    double *xc = (double *)malloc(n * sizeof(double));
    double *xp = (double *)malloc(n * sizeof(double));
    double *y = (double *)malloc(n * sizeof(double));
    double *g = (double *)malloc(n * sizeof(double));
    double *beta = (double *)malloc((size_t)(iters > 0 ? iters : 1) * sizeof(double));
    orc_beta_table(p->momentum, iters, beta);
    memcpy(xc, x0, n * sizeof(double));
    memcpy(xp, x0, n * sizeof(double));
    long long active = 0;
    for (int k = 0; k < iters; k++) {
        for (size_t v = 0; v < n; v++) y[v] = xc[v] + beta[k] * (xc[v] - xp[v]);
        orc_grad_f(p, y, b, w, omtv, g);
        for (size_t v = 0; v < n; v++) {
            double z = y[v] - tau * g[v];
            double t = tau * p->lambda_l1 * (om1 ? om1[v] : 1.0);
            if (fabs(z) > t || t <= 0.0) active++;
            xp[v] = xc[v];
            xc[v] = orc_soft(z, t);
        }
    }
    memcpy(xK, xc, n * sizeof(double));
    free(xc);
    free(xp);
    free(y);
    free(g);
    free(beta);
    return active;
}

/* K steps as orc_unrolled, counting the two places where the unrolled map has
 * a kink: soft-threshold passes (Eq. 21: |z| > t) and voxel-steps on the
 * quadratic branch of the smoothed norm (Eq. 14/16: |Dy| < mu, where the
 * second derivative of h_mu jumps). counts = {passes, quadratic-branch
 * voxel-steps}. Two runs with equal counts take the same branches unless
 * entries and exits cancel. */
void orc_unrolled_counts(const orc_params *p, const double *b, const double *w, const double *om1,
                         const double *omtv, double tau, int iters, const double *x0, double *xK,
                         long long counts[2])
{
    const size_t n = NVOX(p);
    double *xc = (double *)malloc(n * sizeof(double));
    double *xp = (double *)malloc(n * sizeof(double));
    double *y = (double *)malloc(n * sizeof(double));
    double *g = (double *)malloc(n * sizeof(double));
    double *dy = (double *)malloc(3 * n * sizeof(double));
    double *beta = (double *)malloc((size_t)(iters > 0 ? iters : 1) * sizeof(double));
    orc_beta_table(p->momentum, iters, beta);
    memcpy(xc, x0, n * sizeof(double));
    memcpy(xp, x0, n * sizeof(double));
    long long passes = 0, quad = 0;
    for (int k = 0; k < iters; k++) {
        for (size_t v = 0; v < n; v++) y[v] = xc[v] + beta[k] * (xc[v] - xp[v]);
        orc_grad(p, y, dy);
        for (size_t v = 0; v < n; v++) {
            const double s2 = dy[v] * dy[v] + dy[n + v] * dy[n + v] + dy[2 * n + v] * dy[2 * n + v];
            if (sqrt(s2) < p->mu) quad++;
        }
        orc_grad_f(p, y, b, w, omtv, g);
        for (size_t v = 0; v < n; v++) {
            double z = y[v] - tau * g[v];
            double t = tau * p->lambda_l1 * (om1 ? om1[v] : 1.0);
            if (fabs(z) > t || t <= 0.0) passes++;
            xp[v] = xc[v];
            xc[v] = orc_soft(z, t);
        }
    }
    memcpy(xK, xc, n * sizeof(double));
    counts[0] = passes;
    counts[1] = quad;
    free(xc);
    free(xp);
    free(y);
    free(g);
    free(dy);
    free(beta);
}

/* ---------- strong-convexity certificate ---------- */

/* |r|^2 with r = grad f(x+) - grad f(y) + (y - x+)/tau, an element of the
 * subdifferential of F at x+ = prox(y - tau grad f(y)). */
double orc_certificate(const orc_params *p, const double *y, const double *xplus, double tau,
                       const double *b, const double *w, const double *omtv)
{
    const size_t n = NVOX(p);
    double *gy = (double *)malloc(n * sizeof(double));
    double *gx = (double *)malloc(n * sizeof(double));
    orc_grad_f(p, y, b, w, omtv, gy);
    orc_grad_f(p, xplus, b, w, omtv, gx);
    double *pz = (double *)calloc((size_t)p->nz, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++) {
        double s = 0.0;
        for (size_t v = (size_t)z * p->nx * p->ny; v < (size_t)(z + 1) * p->nx * p->ny; v++) {
            double r = gx[v] - gy[v] + (y[v] - xplus[v]) / tau;
            s += r * r;
        }
        pz[z] = s;
    }
    double s = 0.0;
    for (int z = 0; z < p->nz; z++) s += pz[z];
    free(gy);
    free(gx);
    free(pz);
    return s;
}

/* ---------- single-voxel evaluation (for sampled checks at full size) ---------- */

static double y_at(const orc_params *p, const double *xk, const double *xkm1, double beta,
                   int x, int y, int z)
{
    size_t v = AT(p, x, y, z);
    return xk[v] + beta * (xk[v] - xkm1[v]);
}

/* omtv * grad h_mu(D y) at voxel q, component a; zero outside the volume. */
static double p_at(const orc_params *p, const double *xk, const double *xkm1, double beta,
                   const double *omtv, int x, int y, int z, int a)
{
    if (x < 0 || y < 0 || z < 0 || x >= p->nx || y >= p->ny || z >= p->nz) return 0.0;
    double c = y_at(p, xk, xkm1, beta, x, y, z);
    double d0 = x >= 1 ? c - y_at(p, xk, xkm1, beta, x - 1, y, z) : 0.0;
    double d1 = y >= 1 ? c - y_at(p, xk, xkm1, beta, x, y - 1, z) : 0.0;
    double d2 = z >= 1 ? c - y_at(p, xk, xkm1, beta, x, y, z - 1) : 0.0;
    double u[3];
    orc_huber_grad(d0, d1, d2, p->mu, u);
    return (omtv ? omtv[AT(p, x, y, z)] : 1.0) * u[a];
}

/* x_{k+1} at the listed voxels (flat indices), each evaluated from Eq. 17 and
 * Eq. 20-21 directly around that voxel. */
void orc_step_sampled(const orc_params *p, const double *xk, const double *xkm1, double beta,
                      double tau, const double *b, const double *w, const double *om1,
                      const double *omtv, int64_t nsample, const int64_t *idx, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsample; s++) {
        int64_t v = idx[s];
        int x = (int)(v % p->nx);
        int y = (int)((v / p->nx) % p->ny);
        int z = (int)(v / ((int64_t)p->nx * p->ny));
        double div = 0.0;
        if (x >= 1) div += p_at(p, xk, xkm1, beta, omtv, x, y, z, 0);
        div -= p_at(p, xk, xkm1, beta, omtv, x + 1, y, z, 0);
        if (y >= 1) div += p_at(p, xk, xkm1, beta, omtv, x, y, z, 1);
        div -= p_at(p, xk, xkm1, beta, omtv, x, y + 1, z, 1);
        if (z >= 1) div += p_at(p, xk, xkm1, beta, omtv, x, y, z, 2);
        div -= p_at(p, xk, xkm1, beta, omtv, x, y, z + 1, 2);
        double yv = y_at(p, xk, xkm1, beta, x, y, z);
        double g = w[v] * (yv - b[v]) + p->lambda_tv * div;
        out[s] = orc_soft(yv - tau * g, tau * p->lambda_l1 * (om1 ? om1[v] : 1.0));
    }
}

/* ---------- adjoint of K unrolled steps (one round, fixed weights and tau) ---------- */

/* Given gK = dLoss/dx_K, accumulate dLoss/db (gb), dLoss/dw (gw) and
 * gscal = {dLoss/dlambda_l1, dLoss/dlambda_tv}; tau and the weights are held
 * fixed. Forward iterates are stored in full (this is a slow reference). */
int orc_backward(const orc_params *p, const double *b, const double *w, const double *om1,
                 const double *omtv, double tau, int iters, const double *x0, const double *gK,
                 double *gb, double *gw, double gscal[2])
{
    const size_t n = NVOX(p);
    double *X = (double *)malloc((size_t)(iters + 1) * n * sizeof(double));
    double *beta = (double *)malloc((size_t)(iters > 0 ? iters : 1) * sizeof(double));
    if (!X || !beta) return -1;
    orc_beta_table(p->momentum, iters, beta);
    memcpy(X, x0, n * sizeof(double));
    for (int k = 0; k < iters; k++) {
        const double *xk = X + (size_t)k * n;
        const double *xkm1 = k >= 1 ? X + (size_t)(k - 1) * n : X;
        orc_step(p, xk, xkm1, beta[k], tau, b, w, om1, omtv, X + (size_t)(k + 1) * n);
    }
    double *a_next = (double *)malloc(n * sizeof(double)); /* dL/dx_{k+1} */
    double *a_cur = (double *)calloc(n, sizeof(double));   /* dL/dx_k (partial) */
    double *a_prev = (double *)calloc(n, sizeof(double));  /* dL/dx_{k-1} (partial) */
    double *y = (double *)malloc(n * sizeof(double));
    double *gfy = (double *)malloc(n * sizeof(double));
    double *tvg = (double *)malloc(n * sizeof(double));
    double *m = (double *)malloc(n * sizeof(double));
    double *dy = (double *)malloc(3 * n * sizeof(double));
    double *dm = (double *)malloc(3 * n * sizeof(double));
    double *hv = (double *)malloc(n * sizeof(double));
    memcpy(a_next, gK, n * sizeof(double));
    memset(gb, 0, n * sizeof(double));
    memset(gw, 0, n * sizeof(double));
    gscal[0] = 0.0;
    gscal[1] = 0.0;
    for (int k = iters - 1; k >= 0; k--) {
        const double *xk = X + (size_t)k * n;
        const double *xkm1 = k >= 1 ? X + (size_t)(k - 1) * n : X;
        for (size_t v = 0; v < n; v++) y[v] = xk[v] + beta[k] * (xk[v] - xkm1[v]);
        orc_tv_grad(p, y, omtv, tvg);
        /* m = dL/dz = dL/dx_{k+1} where the soft-threshold passes, 0 where it clips */
        double l1acc = 0.0;
        for (size_t v = 0; v < n; v++) {
            gfy[v] = w[v] * (y[v] - b[v]) + p->lambda_tv * tvg[v];
            double z = y[v] - tau * gfy[v];
            double t = tau * p->lambda_l1 * (om1 ? om1[v] : 1.0);
            double pass = (fabs(z) > t || t <= 0.0) ? 1.0 : 0.0;
            m[v] = a_next[v] * pass;
            double sg = z > 0.0 ? 1.0 : (z < 0.0 ? -1.0 : 0.0);
            l1acc += -tau * (om1 ? om1[v] : 1.0) * sg * m[v];
        }
        gscal[0] += l1acc;
        /* Hessian-vector product of the TV term: D^T(omtv H_mu(Dy) D m) */
        orc_grad(p, y, dy);
        orc_grad(p, m, dm);
        for (size_t v = 0; v < n; v++) {
            double z0 = dy[v], z1 = dy[n + v], z2 = dy[2 * n + v];
            double q0 = dm[v], q1 = dm[n + v], q2 = dm[2 * n + v];
            double s = sqrt(z0 * z0 + z1 * z1 + z2 * z2);
            double om = omtv ? omtv[v] : 1.0;
            double h0, h1, h2;
            if (s <= p->mu) {
                h0 = q0 / p->mu;
                h1 = q1 / p->mu;
                h2 = q2 / p->mu;
            } else {
                double e0 = z0 / s, e1 = z1 / s, e2 = z2 / s;
                double eq = e0 * q0 + e1 * q1 + e2 * q2;
                h0 = (q0 - e0 * eq) / s;
                h1 = (q1 - e1 * eq) / s;
                h2 = (q2 - e2 * eq) / s;
            }
            dm[v] = om * h0;
            dm[n + v] = om * h1;
            dm[2 * n + v] = om * h2;
        }
        orc_div(p, dm, hv);
        double tvacc = 0.0;
        for (size_t v = 0; v < n; v++) {
            double ybar = m[v] - tau * (w[v] * m[v] + p->lambda_tv * hv[v]);
            gb[v] += tau * w[v] * m[v];
            gw[v] += -tau * (y[v] - b[v]) * m[v];
            tvacc += -tau * tvg[v] * m[v];
            a_cur[v] += (1.0 + beta[k]) * ybar;
            if (k >= 1)
                a_prev[v] += -beta[k] * ybar;
            else
                a_cur[v] += -beta[k] * ybar; /* x_{-1} = x_0 */
        }
        gscal[1] += tvacc;
        /* shift: dL/dx_k is complete once step k is reversed */
        double *t = a_next;
        a_next = a_cur;
        a_cur = a_prev;
        a_prev = t;
        memset(a_prev, 0, n * sizeof(double));
    }
    free(X);
    free(beta);
    free(a_next);
    free(a_cur);
    free(a_prev);
    free(y);
    free(gfy);
    free(tvg);
    free(m);
    free(dy);
    free(dm);
    free(hv);
    return 0;
}
