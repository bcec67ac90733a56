/*
 * FP64 CPU oracle of the modified Artificial Retina (arXiv:1709.08610).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench load this file's library.  It shares no source,
 * header, table or helper with the CUDA path, and the CUDA path never calls
 * it.  Everything is plain double arithmetic with libm exp(), written for a
 * reader to check against the paper by eye; OpenMP only splits independent
 * cells / seeds / events across threads and never changes an operation order
 * inside one cell or seed.
 *
 * Notation (Section 2, Eq. 1): hits x_k, pattern theta = (theta0, theta1),
 * residual r_k = h_k - J_k theta (the hit minus the track's prediction in the
 * hit's detector plane), s^2 = |r_k|^2,
 *     R(theta) = sum_k exp(-s_k^2 / sigma^2).
 * Track models:
 *   model 0, the 2D toy (Section 2, Figure 1): theta = (alpha, beta),
 *     prediction alpha*x + beta in the plane x = const, so h = y,
 *     J = [x, 1] (1 x 2).
 *   model 1, the simplified VELO (Section 3): theta = (t_x, t_y), a straight
 *     line through the origin crossing the layer z = const at (t_x z, t_y z),
 *     so h = (x, y), J = z * I_2.
 * Derivatives (Section 2, "gradient and Hessian ... small overhead"):
 *     grad R = (2 / sigma^2) sum_k e_k J_k^T r_k
 *     Hess R = sum_k e_k [ (4 / sigma^4) (J_k^T r_k)(J_k^T r_k)^T
 *                          - (2 / sigma^2) J_k^T J_k ].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TOY2D 0
#define OR_VELO_SLOPES 1

typedef struct {
    double lo[2];
    double step[2];
    int64_t n[2];
} or_grid;

/* Residual r (m = 1 or 2 components) and Jacobian rows J (m x 2) of one hit. */
static int hit_residual(const float *hit, int model, const double th[2], double r[2], double J[2][2]) {
    const double x = (double)hit[0], y = (double)hit[1], z = (double)hit[2];
    if (model == OR_TOY2D) {
        J[0][0] = x;
        J[0][1] = 1.0;
        r[0] = y - (th[0] * x + th[1]);
        return 1;
    }
    J[0][0] = z; J[0][1] = 0.0;
    J[1][0] = 0.0; J[1][1] = z;
    r[0] = x - th[0] * z;
    r[1] = y - th[1] * z;
    return 2;
}

/*
 * Eq. 1 with its gradient and Hessian at one theta.
 * out[0] = R, out[1..2] = grad, out[3..5] = (H00, H01, H11),
 * out[6] = sum_k e_k (= R, kept for symmetry),
 * out[7..8] = sum of |gradient terms| per component,
 * out[9..11] = sum of |Hessian terms| per entry (scales for tolerances).
 */
void or_rgh(const float *hits, int64_t n_hits, int model, const double theta[2], double sigma, double *out) {
    const double inv_s2 = 1.0 / (sigma * sigma);
    double R = 0, g0 = 0, g1 = 0, h00 = 0, h01 = 0, h11 = 0;
    double ag0 = 0, ag1 = 0, ah00 = 0, ah01 = 0, ah11 = 0;
    for (int64_t k = 0; k < n_hits; ++k) {
        double r[2], J[2][2];
        const int m = hit_residual(hits + 4 * k, model, theta, r, J);
        double s2 = 0.0;
        for (int a = 0; a < m; ++a) s2 += r[a] * r[a];
        const double e = exp(-s2 * inv_s2);
        /* J^T r and J^T J */
        double jr[2] = {0.0, 0.0}, jj[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int c = 0; c < 2; ++c)
            for (int a = 0; a < m; ++a) jr[c] += J[a][c] * r[a];
        for (int c = 0; c < 2; ++c)
            for (int d = 0; d < 2; ++d)
                for (int a = 0; a < m; ++a) jj[c][d] += J[a][c] * J[a][d];
        const double tg0 = 2.0 * inv_s2 * e * jr[0];
        const double tg1 = 2.0 * inv_s2 * e * jr[1];
        const double t00 = e * (4.0 * inv_s2 * inv_s2 * jr[0] * jr[0] - 2.0 * inv_s2 * jj[0][0]);
        const double t01 = e * (4.0 * inv_s2 * inv_s2 * jr[0] * jr[1] - 2.0 * inv_s2 * jj[0][1]);
        const double t11 = e * (4.0 * inv_s2 * inv_s2 * jr[1] * jr[1] - 2.0 * inv_s2 * jj[1][1]);
        R += e;
        g0 += tg0; g1 += tg1;
        h00 += t00; h01 += t01; h11 += t11;
        ag0 += fabs(tg0); ag1 += fabs(tg1);
        ah00 += fabs(t00); ah01 += fabs(t01); ah11 += fabs(t11);
    }
    out[0] = R; out[1] = g0; out[2] = g1;
    out[3] = h00; out[4] = h01; out[5] = h11;
    out[6] = R; out[7] = ag0; out[8] = ag1;
    out[9] = ah00; out[10] = ah01; out[11] = ah11;
}

/* Eq. 1 alone (no derivatives). */
double or_response(const float *hits, int64_t n_hits, int model, const double theta[2], double sigma) {
    const double inv_s2 = 1.0 / (sigma * sigma);
    double R = 0.0;
    for (int64_t k = 0; k < n_hits; ++k) {
        double r[2], J[2][2];
        const int m = hit_residual(hits + 4 * k, model, theta, r, J);
        double s2 = 0.0;
        for (int a = 0; a < m; ++a) s2 += r[a] * r[a];
        R += exp(-s2 * inv_s2);
    }
    return R;
}

/* Responses at a list of points: R[p] = R(theta_p). */
void or_response_points(const float *hits, int64_t n_hits, int model, const double *theta, int64_t n_pts,
                        double sigma, double *R) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n_pts; ++p) R[p] = or_response(hits, n_hits, model, theta + 2 * p, sigma);
}

/* Grid of units (Eq. 2, step 2 of the grid algorithm): R[i1][i0] = R(theta_{i0 i1}),
 * cell centres theta_a = lo_a + (i_a + 1/2) step_a. */
void or_grid_response(const float *hits, int64_t n_hits, int model, const or_grid *g, double sigma, double *R) {
    const int64_t n0 = g->n[0], n1 = g->n[1];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i1 = 0; i1 < n1; ++i1) {
        for (int64_t i0 = 0; i0 < n0; ++i0) {
            double th[2];
            th[0] = g->lo[0] + ((double)i0 + 0.5) * g->step[0];
            th[1] = g->lo[1] + ((double)i1 + 0.5) * g->step[1];
            R[i1 * n0 + i0] = or_response(hits, n_hits, model, th, sigma);
        }
    }
}

/*
 * Cluster selection on the grid (steps 3-4 of the grid algorithm): a unit is
 * selected when its response is at least R0 and it beats every existing
 * neighbour of its 3 x 3 neighbourhood in the order (R, -linear index), i.e.
 * a strict local maximum with ties going to the lower linear index.  Writes
 * the linear indices (i1 * n0 + i0) of the selected units in increasing
 * order; returns how many there are (which may exceed cap; only cap are
 * written).  margin_out (nullable, one per unit) receives, for every unit,
 * min over its comparisons of |R - R_other| (including R - R0): the distance
 * of that unit's decision from a tie.
 */
int64_t or_grid_maxima(const double *R, int64_t n0, int64_t n1, double R0, int64_t *idx_out, int64_t cap,
                       double *margin_out) {
    int64_t count = 0;
    for (int64_t i1 = 0; i1 < n1; ++i1) {
        for (int64_t i0 = 0; i0 < n0; ++i0) {
            const int64_t lin = i1 * n0 + i0;
            const double v = R[lin];
            int is_max = v >= R0;
            double margin = fabs(v - R0);
            for (int d1 = -1; d1 <= 1; ++d1) {
                for (int d0 = -1; d0 <= 1; ++d0) {
                    if (d0 == 0 && d1 == 0) continue;
                    const int64_t j0 = i0 + d0, j1 = i1 + d1;
                    if (j0 < 0 || j0 >= n0 || j1 < 0 || j1 >= n1) continue;
                    const int64_t nb = j1 * n0 + j0;
                    const double w = R[nb];
                    const int beats = (v > w) || (v == w && lin < nb);
                    if (!beats) is_max = 0;
                    if (fabs(v - w) < margin) margin = fabs(v - w);
                }
            }
            if (margin_out) margin_out[lin] = margin;
            if (is_max) {
                if (count < cap) idx_out[count] = lin;
                ++count;
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Local search: Algorithm 1 with the truncated Newton update (Section 3).    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t q;               /* number of updates per seed (Section 2: fixed count) */
    double sigma[8];         /* bandwidth used at update j (Section 3: annealed)    */
    double c1;               /* Armijo sufficient-increase constant                 */
    int32_t max_halvings;    /* backtracking halvings after the unit step           */
    double step_cap_cells;   /* cap on ||p / step||_inf, in grid cells              */
    int32_t update;          /* direction: 0 truncated Newton, 1 steepest ascent,    */
                             /* 2 Newton with a shifted (modified) Hessian          */
} or_ls_opts;

/*
 * Perturbed replicas of a search (path conditioning; test infrastructure).
 * A search whose discrete decisions all clear their thresholds can still
 * end at a point that float32 arithmetic cannot pin down: a step that solves
 * a badly conditioned system (the shifted modified-Newton step has
 * condition >= 1e3) or a long walk along a flat ridge amplifies the rounding
 * of the sums it uses.  To tell such paths apart the oracle can rerun a seed
 * with every quantity the CUDA path computes in float32 - R, the gradient and
 * the Hessian at each update, R at each line-search trial - displaced by
 * level * u times its parity tolerance (R: 1e-5 |R| + 1e-6; gradient and
 * Hessian entries: 1e-4 of the sum of the absolute values of their terms),
 * with u in [-1, 1) drawn for each (replica key, seed, update, quantity) from
 * the SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014).  A path is
 * well conditioned when such replicas end where the unperturbed one ends.
 * level = 0 reproduces the plain search bit for bit.
 */
typedef struct {
    double level;
    uint64_t key;
} or_perturb;

/* SplitMix64: the state advances by the golden-ratio increment and the
 * output is the state passed through the published 64-bit finaliser. */
uint64_t or_splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* u in [-1, 1) for quantity c of update j of seed i under replica key. */
double or_perturb_u(uint64_t key, int64_t i, int j, int c) {
    uint64_t st = key;
    const uint64_t a = or_splitmix64(&st);
    st = a ^ ((uint64_t)i * 0x100000ULL + (uint64_t)j * 0x100ULL + (uint64_t)c);
    const uint64_t h = or_splitmix64(&st);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* quantity indices: 0 R, 1-2 gradient, 3-5 Hessian (00 01 11), 16 + h trial h's R */
static double perturbed(const or_perturb *pt, int64_t i, int j, int c, double v, double tol) {
    if (!pt || pt->level == 0.0) return v;
    return v + pt->level * tol * or_perturb_u(pt->key, i, j, c);
}

/*
 * One truncated Newton direction (Newton-CG, Nocedal & Wright Alg. 7.1)
 * for maximising R, i.e. minimising f = -R with gradient -g and Hessian
 * B = -H.  CG on B p = g from p = 0, forcing tolerance
 * eps = min(1/2, sqrt(|g|)) |g|, stopping at negative curvature (first
 * iteration: fall back to the steepest-ascent direction g) and after at
 * most 2 iterations (the dimension).  *margin gets the smallest distance of
 * a branch test from its threshold, in units of the FP32 parity tolerance
 * of the quantities compared: 1e-4 of the sum of absolute terms plus the
 * absolute floor of each gradient (gfloor) or Hessian (hfloor) entry.
 */
static void newton_cg_direction(const double g[2], const double H[3], const double gabs[2],
                                const double Habs[3], double gfloor, double hfloor, double p[2], double *margin) {
    const double B00 = -H[0], B01 = -H[1], B11 = -H[2];
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1]);
    const double eps = fmin(0.5, sqrt(gn)) * gn;
    double z[2] = {0.0, 0.0};
    double r[2] = {-g[0], -g[1]};   /* residual of B z = g at z = 0, as B z - g */
    double d[2] = {g[0], g[1]};
    const double hscale = Habs[0] + 2.0 * Habs[1] + Habs[2];
    for (int it = 0; it < 2; ++it) {
        const double Bd0 = B00 * d[0] + B01 * d[1];
        const double Bd1 = B01 * d[0] + B11 * d[1];
        const double dBd = d[0] * Bd0 + d[1] * Bd1;
        const double dd = d[0] * d[0] + d[1] * d[1];
        {
            const double tol = (1e-4 * hscale + 4.0 * hfloor) * dd;
            const double m = tol > 0.0 ? fabs(dBd) / tol : 0.0;
            if (m < *margin) *margin = m;
        }
        if (dBd <= 0.0) {
            if (it == 0) { p[0] = g[0]; p[1] = g[1]; }
            else { p[0] = z[0]; p[1] = z[1]; }
            return;
        }
        const double rr = r[0] * r[0] + r[1] * r[1];
        const double alpha = rr / dBd;
        z[0] += alpha * d[0];
        z[1] += alpha * d[1];
        double rn[2] = {r[0] + alpha * Bd0, r[1] + alpha * Bd1};
        const double rnn = sqrt(rn[0] * rn[0] + rn[1] * rn[1]);
        if (it == 0) {
            const double tol = 1e-4 * (gabs[0] + gabs[1]) + 2.0 * gfloor;
            const double m = tol > 0.0 ? fabs(rnn - eps) / tol : 0.0;
            if (m < *margin) *margin = m;
        }
        if (rnn < eps) { p[0] = z[0]; p[1] = z[1]; return; }
        const double beta = (rn[0] * rn[0] + rn[1] * rn[1]) / rr;
        d[0] = -rn[0] + beta * d[0];
        d[1] = -rn[1] + beta * d[1];
        r[0] = rn[0];
        r[1] = rn[1];
    }
    p[0] = z[0];
    p[1] = z[1];
}

/*
 * Newton direction with a modified Hessian (Nocedal & Wright, Section 3.4):
 * B = -H is shifted by tau I, tau = max(0, delta - mu1), mu1 <= mu2 the
 * eigenvalues of B and delta = 1e-3 max(|mu1|, |mu2|), so that B + tau I is
 * positive definite with smallest eigenvalue >= delta; p solves
 * (B + tau I) p = g.  Where -H is already positive definite beyond delta this
 * is the plain Newton step.  B = 0 (no curvature) gives p = g.  *margin gets
 * the distance of the shift test mu1 < delta from its threshold, in units of
 * 1e-4 of the sum of absolute Hessian terms plus each entry's absolute floor
 * hfloor.  A shifted step is otherwise an
 * ordinary decision: B + tau I then has condition number >= 1e3, so the
 * direction can move by more than the Hessian tolerance bounds; whether that
 * changes where the path ends is what the perturbed replicas measure.
 */
static void modified_newton_direction(const double g[2], const double H[3], const double Habs[3], double hfloor,
                                      double p[2], double *margin) {
    const double a = -H[0], b = -H[1], c = -H[2];
    const double mid = 0.5 * (a + c), rad = sqrt(0.25 * (a - c) * (a - c) + b * b);
    const double mu1 = mid - rad, mu2 = mid + rad;
    const double delta = 1e-3 * fmax(fabs(mu1), fabs(mu2));
    {
        const double tol = 1e-4 * (Habs[0] + 2.0 * Habs[1] + Habs[2]) + 4.0 * hfloor;
        const double m = tol > 0.0 ? fabs(mu1 - delta) / tol : 0.0;
        if (m < *margin) *margin = m;
    }
    if (!(delta > 0.0)) {
        p[0] = g[0];
        p[1] = g[1];
        return;
    }
    const double tau = mu1 < delta ? delta - mu1 : 0.0;
    const double a2 = a + tau, c2 = c + tau;
    const double det = a2 * c2 - b * b;
    p[0] = (c2 * g[0] - b * g[1]) / det;
    p[1] = (a2 * g[1] - b * g[0]) / det;
}

/*
 * One seed through Algorithm 1's q updates.  Returns the status:
 * 0 ok, 1 some line search accepted no step, 2 final point outside the box,
 * 3 non-finite.  *margin receives the smallest distance of any discrete
 * decision (curvature sign, CG stop, Armijo test, box test) from its
 * threshold, in units of the FP32 parity tolerance of the compared values
 * (R: 1e-5 R + 1e-6; gradient / Hessian: 1e-4 of the absolute terms plus
 * floors of 1e-6 of their scale at unit response - one hit at residual
 * sigma: 2 sigma |J|max / sigma^2 for the gradient, 2 |J|max^2 / sigma^2 for
 * the Hessian, |J|max the largest Jacobian entry over the event's hits,
 * jmax - below which float32 sums, whose exponentials flush to zero under
 * 2^-126, carry no information; theta: 1e-3 of a cell), so that callers can
 * tell genuine disagreements from ties (margin < 1).
 */
static int search_one(const float *hits, int64_t n_hits, int model, const float seed[2], const or_ls_opts *o,
                      const or_grid *box, double jmax, double theta_out[2], double *R_out, double *margin,
                      const or_perturb *pt, int64_t seed_index, int32_t *trials) {
    double th[2] = {(double)seed[0], (double)seed[1]};
    int status = 0;
    *margin = INFINITY;
    for (int j = 0; j < o->q; ++j) {
        const double sigma = o->sigma[j];
        double rgh[12];
        or_rgh(hits, n_hits, model, th, sigma, rgh);
        const double gabs[2] = {rgh[7], rgh[8]};
        const double Habs[3] = {rgh[9], rgh[10], rgh[11]};
        const double k = 1.0 / (sigma * sigma);
        const double gfloor = 1e-6 * 2.0 * k * sigma * jmax, hfloor = 1e-6 * 2.0 * k * jmax * jmax;
        const int64_t si = seed_index;
        const double R = perturbed(pt, si, j, 0, rgh[0], 1e-5 * fabs(rgh[0]) + 1e-6);
        const double g[2] = {perturbed(pt, si, j, 1, rgh[1], 1e-4 * gabs[0] + gfloor),
                             perturbed(pt, si, j, 2, rgh[2], 1e-4 * gabs[1] + gfloor)};
        const double H[3] = {perturbed(pt, si, j, 3, rgh[3], 1e-4 * Habs[0] + hfloor),
                             perturbed(pt, si, j, 4, rgh[4], 1e-4 * Habs[1] + hfloor),
                             perturbed(pt, si, j, 5, rgh[5], 1e-4 * Habs[2] + hfloor)};
        double p[2];
        if (o->update == 1) {         /* steepest ascent: the gradient itself */
            p[0] = g[0];
            p[1] = g[1];
        } else if (o->update == 2) {
            modified_newton_direction(g, H, Habs, hfloor, p, margin);
        } else {
            newton_cg_direction(g, H, gabs, Habs, gfloor, hfloor, p, margin);
        }
        /* cap the step length, measured in grid cells */
        const double cells = fmax(fabs(p[0]) / box->step[0], fabs(p[1]) / box->step[1]);
        if (cells > o->step_cap_cells) {
            const double s = o->step_cap_cells / cells;
            p[0] *= s;
            p[1] *= s;
        }
        /* backtracking line search with the Armijo sufficient-increase test */
        const double slope = g[0] * p[0] + g[1] * p[1];
        double t = 1.0;
        int accepted = 0;
        for (int h = 0; h <= o->max_halvings; ++h) {
            const double trial[2] = {th[0] + t * p[0], th[1] + t * p[1]};
            const double Rt0 = or_response(hits, n_hits, model, trial, sigma);
            if (trials) ++*trials;
            const double Rt = perturbed(pt, seed_index, j, 16 + h, Rt0, 1e-5 * fabs(Rt0) + 1e-6);
            const double need = R + o->c1 * t * slope;
            const double tol = 1e-5 * (fabs(R) + fabs(Rt)) + 2e-6;
            const double m = fabs(Rt - need) / tol;
            if (m < *margin) *margin = m;
            if (Rt >= need) {
                th[0] = trial[0];
                th[1] = trial[1];
                accepted = 1;
                break;
            }
            t *= 0.5;
        }
        if (!accepted) status = 1;
    }
    *R_out = or_response(hits, n_hits, model, th, o->sigma[o->q - 1]);
    theta_out[0] = th[0];
    theta_out[1] = th[1];
    if (!(isfinite(th[0]) && isfinite(th[1]) && isfinite(*R_out))) return 3;
    for (int a = 0; a < 2; ++a) {
        const double lo = box->lo[a], hi = box->lo[a] + (double)box->n[a] * box->step[a];
        const double m = fmin(fabs(th[a] - lo), fabs(th[a] - hi)) / (1e-3 * box->step[a]);
        if (m < *margin) *margin = m;
        if (!(th[a] >= lo && th[a] < hi)) return 2;
    }
    return status;
}

/* The largest Jacobian entry over the hits: |z| (slope model) or
 * max(|x|, 1) (2D toy), the scale of the gradient / Hessian floors. */
static double jacobian_max(const float *hits, int64_t n_hits, int model) {
    double m = model == OR_TOY2D ? 1.0 : 0.0;
    for (int64_t k = 0; k < n_hits; ++k) {
        const double v = fabs((double)hits[4 * k + (model == OR_TOY2D ? 0 : 2)]);
        if (v > m) m = v;
    }
    return m;
}

void or_local_search(const float *hits, int64_t n_hits, int model, const float *seeds, int64_t n_seeds,
                     const or_ls_opts *o, const or_grid *box, double *theta_out, double *R_out, uint8_t *status,
                     double *margin_out) {
    const double jmax = jacobian_max(hits, n_hits, model);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_seeds; ++i) {
        double m;
        status[i] = (uint8_t)search_one(hits, n_hits, model, seeds + 2 * i, o, box, jmax, theta_out + 2 * i,
                                        R_out + i, &m, NULL, i, NULL);
        if (margin_out) margin_out[i] = m;
    }
}

/* or_local_search with the perturbation (level, key) applied; seed i draws
 * its displacements under index index_base + i. */
void or_local_search_perturbed(const float *hits, int64_t n_hits, int model, const float *seeds, int64_t n_seeds,
                               const or_ls_opts *o, const or_grid *box, double level, uint64_t key,
                               int64_t index_base, double *theta_out, double *R_out, uint8_t *status,
                               double *margin_out) {
    const or_perturb pt = {level, key};
    const double jmax = jacobian_max(hits, n_hits, model);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_seeds; ++i) {
        double m;
        status[i] = (uint8_t)search_one(hits, n_hits, model, seeds + 2 * i, o, box, jmax, theta_out + 2 * i,
                                        R_out + i, &m, &pt, index_base + i, NULL);
        if (margin_out) margin_out[i] = m;
    }
}

/* or_local_search that also counts each seed's line-search trials (the
 * responses evaluated besides the q gradient / Hessian evaluations). */
void or_local_search_counted(const float *hits, int64_t n_hits, int model, const float *seeds, int64_t n_seeds,
                             const or_ls_opts *o, const or_grid *box, double *theta_out, double *R_out,
                             uint8_t *status, int32_t *trials_out) {
    const double jmax = jacobian_max(hits, n_hits, model);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_seeds; ++i) {
        double m;
        trials_out[i] = 0;
        status[i] = (uint8_t)search_one(hits, n_hits, model, seeds + 2 * i, o, box, jmax, theta_out + 2 * i,
                                        R_out + i, &m, NULL, i, trials_out + i);
    }
}

/* ------------------------------------------------------------------------ */
/* Cluster the converged points and keep the best of each (Algorithm 1).     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double R;
    int64_t idx;
} or_rank;

static int rank_cmp(const void *a, const void *b) {
    const or_rank *x = (const or_rank *)a, *y = (const or_rank *)b;
    if (x->R > y->R) return -1;
    if (x->R < y->R) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx) ? 1 : 0;
}

/*
 * Points with status 0 or 1, inside the box [lo, lo + n step) and with
 * R >= R0 are candidates.  They are visited by decreasing R (ties: lower
 * index first); a candidate is kept when, for every point kept before it,
 * max_a |theta_a - theta_kept_a| / step_a >= merge_cells.  Writes the kept
 * point indices in that visiting order; returns how many (may exceed cap).
 * status may be NULL (all 0).
 */
int64_t or_extract_tracks(const double *theta, const double *R, const uint8_t *status, int64_t n_points,
                          const or_grid *box, double R0, double merge_cells, int64_t *keep_out, int64_t cap) {
    or_rank *cand = (or_rank *)malloc(sizeof(or_rank) * (size_t)(n_points > 0 ? n_points : 1));
    int64_t nc = 0;
    for (int64_t i = 0; i < n_points; ++i) {
        if (status && status[i] > 1) continue;
        const double t0 = theta[2 * i], t1 = theta[2 * i + 1];
        if (!(isfinite(t0) && isfinite(t1) && isfinite(R[i]))) continue;
        int inside = 1;
        for (int a = 0; a < 2; ++a) {
            const double v = theta[2 * i + a];
            const double lo = box->lo[a], hi = box->lo[a] + (double)box->n[a] * box->step[a];
            if (!(v >= lo && v < hi)) inside = 0;
        }
        if (!inside || !(R[i] >= R0)) continue;
        cand[nc].R = R[i];
        cand[nc].idx = i;
        ++nc;
    }
    qsort(cand, (size_t)nc, sizeof(or_rank), rank_cmp);
    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t nk = 0;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t i = cand[c].idx;
        int keep = 1;
        for (int64_t k = 0; k < nk && keep; ++k) {
            const int64_t j = kept[k];
            const double d0 = fabs(theta[2 * i] - theta[2 * j]) / box->step[0];
            const double d1 = fabs(theta[2 * i + 1] - theta[2 * j + 1]) / box->step[1];
            if (fmax(d0, d1) < merge_cells) keep = 0;
        }
        if (keep) {
            if (nk < cap) keep_out[nk] = i;
            kept[nk++] = i;
        }
    }
    free(kept);
    free(cand);
    return nk;
}

/* ------------------------------------------------------------------------ */
/* Four-parameter straight track: a line that need not pass through the     */
/* origin, so a vertex displaced along z (or across it) is representable.   */
/*   theta = (x0, y0, t_x, t_y) at a reference plane z_ref: the track crosses */
/*   the layer z at (x0 + t_x w, y0 + t_y w), w = z - z_ref, so               */
/*   r = (x - x0 - t_x w, y - y0 - t_y w) and                                 */
/*   dr/dtheta = -[[1, 0, w, 0], [0, 1, 0, w]]; with J = -dr/dtheta the        */
/*   derivatives of Eq. 1 take the same form as above:                        */
/*     grad R = (2 / sigma^2) sum_k e_k J_k^T r_k                             */
/*     Hess R = sum_k e_k [ (4 / sigma^4) (J_k^T r_k)(J_k^T r_k)^T             */
/*                          - (2 / sigma^2) J_k^T J_k ].                      */
/* z_ref = the layers' mean z makes sum w = 0 over a full track, which        */
/* decouples offsets from slopes in J^T J (the truncated Newton then needs   */
/* a few updates, not tens); z_ref = 0 is the line through the origin's      */
/* parametrisation with two extra offsets.                                  */
/* ------------------------------------------------------------------------ */

/* Upper-triangle index of (a, b), a <= b, in the order 00 01 02 03 11 12 13 22 23 33. */
static int tri4(int a, int b) {
    static const int base[4] = {0, 4, 7, 9};
    return base[a] + (b - a);
}

/*
 * out[0] = R, out[1..4] = grad, out[5..14] = Hess (upper triangle, tri4
 * order), out[15..18] = sum of |gradient terms|, out[19..28] = sum of
 * |Hessian terms| (the scales of the FP32 parity tolerances).
 */
void or_rgh4(const float *hits, int64_t n_hits, const double th[4], double zref, double sigma, double *out) {
    const double k = 1.0 / (sigma * sigma);
    memset(out, 0, sizeof(double) * 29);
    for (int64_t i = 0; i < n_hits; ++i) {
        const float *h = hits + 4 * i;
        const double z = (double)h[2] - zref;
        const double r[2] = {(double)h[0] - th[0] - th[2] * z, (double)h[1] - th[1] - th[3] * z};
        const double e = exp(-(r[0] * r[0] + r[1] * r[1]) * k);
        /* J^T r and J^T J with J = [[1, 0, z, 0], [0, 1, 0, z]] */
        const double Jr[4] = {r[0], r[1], z * r[0], z * r[1]};
        double JJ[4][4] = {{1.0, 0.0, z, 0.0}, {0.0, 1.0, 0.0, z}, {z, 0.0, z * z, 0.0}, {0.0, z, 0.0, z * z}};
        out[0] += e;
        for (int a = 0; a < 4; ++a) {
            const double t = 2.0 * k * e * Jr[a];
            out[1 + a] += t;
            out[15 + a] += fabs(t);
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a; b < 4; ++b) {
                const double t1 = 4.0 * k * k * e * Jr[a] * Jr[b];
                const double t2 = 2.0 * k * e * JJ[a][b];
                out[5 + tri4(a, b)] += t1 - t2;
                out[19 + tri4(a, b)] += fabs(t1) + fabs(t2);
            }
    }
}

double or_response4(const float *hits, int64_t n_hits, const double th[4], double zref, double sigma) {
    const double k = 1.0 / (sigma * sigma);
    double R = 0.0;
    for (int64_t i = 0; i < n_hits; ++i) {
        const float *h = hits + 4 * i;
        const double z = (double)h[2] - zref;
        const double r0 = (double)h[0] - th[0] - th[2] * z, r1 = (double)h[1] - th[1] - th[3] * z;
        R += exp(-(r0 * r0 + r1 * r1) * k);
    }
    return R;
}

typedef struct {
    int32_t q;             /* updates per seed                                   */
    double sigma[8];       /* bandwidth at update j                              */
    double c1;             /* Armijo sufficient-increase constant                */
    int32_t max_halvings;  /* backtracking halvings after the unit step          */
    double scale[4];       /* unit of each parameter for the step cap            */
    double step_cap;       /* cap on max_a |p_a| / scale_a                        */
    double zref;           /* reference plane of the offsets                      */
} or_ls4_opts;

static double sym4(const double *Hu, int a, int b) { return a <= b ? Hu[tri4(a, b)] : Hu[tri4(b, a)]; }

/*
 * Newton-CG direction in four dimensions (Nocedal & Wright, Algorithm 7.1)
 * for maximising R, in the variables scaled by the parameters' units D =
 * diag(scale) (offsets in mm and slopes differ by three orders of
 * magnitude; unscaled, the forcing term stops CG before the offsets move):
 * CG on (D B D) y = D g with B = -Hess R from y = 0, forcing tolerance
 * min(1/2, sqrt|D g|) |D g|, at most 4 iterations (the dimension);
 * non-positive curvature along d returns y = D g at the first iteration,
 * else the current iterate; p = D y.  *margin as for the 2D direction, on
 * the scaled quantities (gfloor, hfloor: the absolute floors of the gradient
 * and Hessian entries, hfloor in tri4 order).
 */
static void newton_cg_direction4(const double g_in[4], const double Hu[10], const double gabs_in[4],
                                 const double Habs[10], const double gfloor[4], const double hfloor[10],
                                 const double scale[4], double p[4], double *margin) {
    double B[4][4], g[4], hscale = 0.0, gsum = 0.0;
    for (int a = 0; a < 4; ++a) {
        g[a] = scale[a] * g_in[a];
        gsum += scale[a] * (gabs_in[a] + 1e4 * gfloor[a]);
        for (int b = 0; b < 4; ++b) {
            B[a][b] = -scale[a] * sym4(Hu, a, b) * scale[b];
            hscale += scale[a] * (sym4(Habs, a, b) + 1e4 * sym4(hfloor, a, b)) * scale[b];
        }
    }
    double gn = 0.0;
    for (int a = 0; a < 4; ++a) gn += g[a] * g[a];
    gn = sqrt(gn);
    const double eps = fmin(0.5, sqrt(gn)) * gn;
    double z[4] = {0, 0, 0, 0}, r[4], d[4];
    for (int a = 0; a < 4; ++a) {
        r[a] = -g[a];
        d[a] = g[a];
    }
    for (int it = 0; it < 4; ++it) {
        double Bd[4], dBd = 0.0, dd = 0.0;
        for (int a = 0; a < 4; ++a) {
            Bd[a] = 0.0;
            for (int b = 0; b < 4; ++b) Bd[a] += B[a][b] * d[b];
            dBd += d[a] * Bd[a];
            dd += d[a] * d[a];
        }
        {
            const double tol = 1e-4 * hscale * dd;
            const double m = tol > 0.0 ? fabs(dBd) / tol : 0.0;
            if (m < *margin) *margin = m;
        }
        if (dBd <= 0.0) {
            for (int a = 0; a < 4; ++a) p[a] = scale[a] * (it == 0 ? g[a] : z[a]);
            return;
        }
        double rr = 0.0;
        for (int a = 0; a < 4; ++a) rr += r[a] * r[a];
        const double alpha = rr / dBd;
        double rn[4], rnn2 = 0.0;
        for (int a = 0; a < 4; ++a) {
            z[a] += alpha * d[a];
            rn[a] = r[a] + alpha * Bd[a];
            rnn2 += rn[a] * rn[a];
        }
        {
            const double tol = 1e-4 * gsum;
            const double m = tol > 0.0 ? fabs(sqrt(rnn2) - eps) / tol : 0.0;
            if (m < *margin) *margin = m;
        }
        if (sqrt(rnn2) < eps) break;
        const double beta = rnn2 / rr;
        for (int a = 0; a < 4; ++a) {
            d[a] = -rn[a] + beta * d[a];
            r[a] = rn[a];
        }
    }
    for (int a = 0; a < 4; ++a) p[a] = scale[a] * z[a];
}

/*
 * Algorithm 1's q updates for one four-parameter seed (float32 start):
 * Newton-CG direction, step cap max_a |p_a| / scale_a <= step_cap, Armijo
 * backtracking; pt (nullable) displaces R, the gradient, the Hessian and
 * the trial responses as for the two-parameter search (quantities 0 R,
 * 1-4 gradient, 5-14 Hessian, 32 + h trial h).  Returns the status: 0 ok,
 * 1 some line search accepted no step, 3 non-finite.
 */
static int search4_one(const float *hits, int64_t n_hits, const float *seed, const or_ls4_opts *o,
                       const or_perturb *pt, int64_t si, double th[4], double *R_out, double *margin) {
    int st = 0;
    *margin = INFINITY;
    /* the largest Jacobian entry per parameter: 1 for the offsets, |z - zref| for the slopes */
    double jm[4] = {1.0, 1.0, 0.0, 0.0};
    for (int64_t k = 0; k < n_hits; ++k) {
        const double w = fabs((double)hits[4 * k + 2] - o->zref);
        if (w > jm[2]) jm[2] = jm[3] = w;
    }
    for (int a = 0; a < 4; ++a) th[a] = (double)seed[a];
    for (int j = 0; j < o->q; ++j) {
        const double sigma = o->sigma[j];
        const double k = 1.0 / (sigma * sigma);
        double gfloor[4], hfloor[10];
        for (int a = 0; a < 4; ++a) {
            gfloor[a] = 1e-6 * 2.0 * k * sigma * jm[a];
            for (int b = a; b < 4; ++b) hfloor[tri4(a, b)] = 1e-6 * 2.0 * k * jm[a] * jm[b];
        }
        double v[29];
        or_rgh4(hits, n_hits, th, o->zref, sigma, v);
        v[0] = perturbed(pt, si, j, 0, v[0], 1e-5 * fabs(v[0]) + 1e-6);
        for (int a = 0; a < 4; ++a) v[1 + a] = perturbed(pt, si, j, 1 + a, v[1 + a], 1e-4 * v[15 + a] + gfloor[a]);
        for (int e = 0; e < 10; ++e) v[5 + e] = perturbed(pt, si, j, 5 + e, v[5 + e], 1e-4 * v[19 + e] + hfloor[e]);
        const double R = v[0];
        double p[4];
        newton_cg_direction4(v + 1, v + 5, v + 15, v + 19, gfloor, hfloor, o->scale, p, margin);
        double cells = 0.0;
        for (int a = 0; a < 4; ++a) cells = fmax(cells, fabs(p[a]) / o->scale[a]);
        if (cells > o->step_cap)
            for (int a = 0; a < 4; ++a) p[a] *= o->step_cap / cells;
        double slope = 0.0;
        for (int a = 0; a < 4; ++a) slope += v[1 + a] * p[a];
        double t = 1.0;
        int accepted = 0;
        for (int hv = 0; hv <= o->max_halvings; ++hv) {
            double trial[4];
            for (int a = 0; a < 4; ++a) trial[a] = th[a] + t * p[a];
            const double Rt0 = or_response4(hits, n_hits, trial, o->zref, sigma);
            const double Rt = perturbed(pt, si, j, 32 + hv, Rt0, 1e-5 * fabs(Rt0) + 1e-6);
            const double need = R + o->c1 * t * slope;
            const double tol = 1e-5 * (fabs(R) + fabs(Rt)) + 2e-6;
            const double m = fabs(Rt - need) / tol;
            if (m < *margin) *margin = m;
            if (Rt >= need) {
                for (int a = 0; a < 4; ++a) th[a] = trial[a];
                accepted = 1;
                break;
            }
            t *= 0.5;
        }
        if (!accepted) st = 1;
    }
    *R_out = or_response4(hits, n_hits, th, o->zref, o->sigma[o->q - 1]);
    int finite = isfinite(*R_out);
    for (int a = 0; a < 4; ++a) finite = finite && isfinite(th[a]);
    return finite ? st : 3;
}

/*
 * Algorithm 1's q updates for four-parameter seeds [n][4]; R_out =
 * R(theta_q; sigma_q); margin as in or_local_search.
 */
void or_local_search4(const float *hits, int64_t n_hits, const float *seeds, int64_t n_seeds, const or_ls4_opts *o,
                      double *theta_out, double *R_out, uint8_t *status, double *margin_out) {
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_seeds; ++i) {
        double m;
        status[i] = (uint8_t)search4_one(hits, n_hits, seeds + 4 * i, o, NULL, i, theta_out + 4 * i, R_out + i, &m);
        if (margin_out) margin_out[i] = m;
    }
}

/* or_local_search4 with the perturbation (level, key); seed i draws under
 * index index_base + i. */
void or_local_search4_perturbed(const float *hits, int64_t n_hits, const float *seeds, int64_t n_seeds,
                                const or_ls4_opts *o, double level, uint64_t key, int64_t index_base,
                                double *theta_out, double *R_out, uint8_t *status, double *margin_out) {
    const or_perturb pt = {level, key};
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_seeds; ++i) {
        double m;
        status[i] = (uint8_t)search4_one(hits, n_hits, seeds + 4 * i, o, &pt, index_base + i, theta_out + 4 * i,
                                         R_out + i, &m);
        if (margin_out) margin_out[i] = m;
    }
}

/* ------------------------------------------------------------------------ */
/* Starting points of the four-parameter search from pairs of hits (our    */
/* reading; the paper leaves the prior P_theta open and has no four-       */
/* parameter search).  Every track comes from the beam line, so a pair of  */
/* its hits on two layers spans a line that passes close to the z axis    */
/* inside the luminous region; a pair of hits from different tracks rarely */
/* does.  The decisions are taken in float32 with one rounding per         */
/* operation, in the order written (the CUDA path takes them the same way, */
/* so that the same pairs are kept on both sides).                         */
/* ------------------------------------------------------------------------ */

/*
 * For each layer pair p (z_a = layer_z[2 p], z_b = layer_z[2 p + 1]), in
 * order, every hit i with |z_i - z_a| <= dz_tol and every hit j with
 * |z_j - z_b| <= dz_tol, both in increasing index order (i outer): the line
 * through h_i and h_j has slopes t = (x_j - x_i, y_j - y_i) / (z_j - z_i);
 * its transverse distance to the z axis is |x_i t_y - y_i t_x| / |t| and it
 * comes closest at z_c = z_i - (x_i t_x + y_i t_y) / |t|^2.  The pair is kept
 * when |t|^2 > 0, (x_i t_y - y_i t_x)^2 <= d_max^2 |t|^2 and
 * zc_lo <= z_c <= zc_hi; its seed is (x0, y0, t_x, t_y) at zref,
 * x0 = x_i + t_x (zref - z_i).  Writes the first `cap` seeds [cap][4] in
 * that order; returns how many pairs were kept (may exceed cap).
 */
int64_t or_pair_seeds4(const float *hits, int64_t n_hits, const float *layer_z, int32_t n_pairs, float dz_tol,
                       float d_max, float zc_lo, float zc_hi, float zref, float *seeds_out, int64_t cap) {
    int64_t count = 0;
    const float dm2 = d_max * d_max;
    for (int32_t p = 0; p < n_pairs; ++p) {
        const float za = layer_z[2 * p], zb = layer_z[2 * p + 1];
        for (int64_t i = 0; i < n_hits; ++i) {
            const float xi = hits[4 * i], yi = hits[4 * i + 1], zi = hits[4 * i + 2];
            if (!(fabsf(zi - za) <= dz_tol)) continue;
            for (int64_t j = 0; j < n_hits; ++j) {
                const float xj = hits[4 * j], yj = hits[4 * j + 1], zj = hits[4 * j + 2];
                if (!(fabsf(zj - zb) <= dz_tol)) continue;
                const float dz = zj - zi;
                const float tx = (xj - xi) / dz;
                const float ty = (yj - yi) / dz;
                const float txx = tx * tx, tyy = ty * ty;
                const float tt = txx + tyy;
                if (!(tt > 0.0f)) continue;
                const float cp = xi * ty, cq = yi * tx;
                const float c = cp - cq;
                const float lhs = c * c, rhs = dm2 * tt;
                if (!(lhs <= rhs)) continue;
                const float ua = xi * tx, ub = yi * ty;
                const float u = ua + ub;
                const float zc = zi - u / tt;
                if (!(zc >= zc_lo && zc <= zc_hi)) continue;
                if (count < cap) {
                    const float w = zref - zi;
                    const float px = tx * w, py = ty * w;
                    seeds_out[4 * count] = xi + px;
                    seeds_out[4 * count + 1] = yi + py;
                    seeds_out[4 * count + 2] = tx;
                    seeds_out[4 * count + 3] = ty;
                }
                ++count;
            }
        }
    }
    return count;
}

/*
 * Cluster / select for four-parameter points (the last two lines of
 * Algorithm 1 with theta = (x0, y0, t_x, t_y)): points with status 0 or 1,
 * finite, slopes inside the slope box [lo, lo + n step) and R >= R0 are
 * candidates, visited by decreasing R (ties: lower index first); a candidate
 * is kept when, for every point kept before it,
 * max_a |theta_a - theta_kept_a| / unit_a >= merge_units.  Writes the kept
 * indices in that order (first cap of them); returns how many were kept.
 */
int64_t or_extract_tracks4(const double *theta, const double *R, const uint8_t *status, int64_t n_points,
                           const or_grid *slope_box, const double unit[4], double R0, double merge_units,
                           int64_t *keep_out, int64_t cap) {
    or_rank *cand = (or_rank *)malloc(sizeof(or_rank) * (size_t)(n_points > 0 ? n_points : 1));
    int64_t nc = 0;
    for (int64_t i = 0; i < n_points; ++i) {
        if (status && status[i] > 1) continue;
        int ok = isfinite(R[i]);
        for (int a = 0; a < 4; ++a) ok = ok && isfinite(theta[4 * i + a]);
        if (!ok) continue;
        for (int a = 0; a < 2; ++a) {
            const double v = theta[4 * i + 2 + a];
            const double lo = slope_box->lo[a], hi = slope_box->lo[a] + (double)slope_box->n[a] * slope_box->step[a];
            if (!(v >= lo && v < hi)) ok = 0;
        }
        if (!ok || !(R[i] >= R0)) continue;
        cand[nc].R = R[i];
        cand[nc].idx = i;
        ++nc;
    }
    qsort(cand, (size_t)nc, sizeof(or_rank), rank_cmp);
    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t nk = 0;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t i = cand[c].idx;
        int keep = 1;
        for (int64_t k = 0; k < nk && keep; ++k) {
            const int64_t j = kept[k];
            double d = 0.0;
            for (int a = 0; a < 4; ++a) d = fmax(d, fabs(theta[4 * i + a] - theta[4 * j + a]) / unit[a]);
            if (d < merge_units) keep = 0;
        }
        if (keep) {
            if (nk < cap) keep_out[nk] = i;
            kept[nk++] = i;
        }
    }
    free(kept);
    free(cand);
    return nk;
}
