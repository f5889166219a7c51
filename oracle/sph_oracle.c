/*
 * sph_oracle.c -- the CPU oracle of the SPH cell-pair offload pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it, and the two share no
 * code, headers or tables.
 *
 * What it computes, plainly and slowly, in FP64:
 *
 *   - the cubic-spline (M4) kernel with compact support H = kernel_gamma * h
 *     (normalisation 8/pi for support H, so that its volume integral is 1);
 *   - the three interaction loops of Sec. 2.1 (density, gradient, force, in
 *     that order) and the linear "ghost" update between density and gradient
 *     (Sec. 2.1 mentions these linear kernels), by brute-force O(N^2)
 *     minimum-image neighbour search in a periodic box.  The SPH forms are the
 *     density-energy formulation with grad-h terms, a Monaghan signal-velocity
 *     viscosity with a Balsara switch and artificial conduction, i.e. the
 *     Sphenix family the paper names in Sec. 2.1;
 *   - the cell grid (Sec. 2.2: cells no smaller than the largest support), the
 *     self + pair task list with periodic shifts, bundles of consecutive tasks
 *     (Sec. 2.3), and byte-exact definitions of pack (gather of a loop's view,
 *     Table 1, with the periodic shift applied to positions, Sec. 2.3) and
 *     unpack (ordered reduction of per-slot results into the particles,
 *     Sec. 2.3);
 *   - the particle-store layouts of Sec. 3.1 (AoS, random-order AoS, the sAoS
 *     pack-gradient / pack-force / pack-shared splits, their by-type splits,
 *     and SoA) as byte images.
 *
 * Per-particle physics is evaluated for a selection of particles so that
 * large workloads can be checked on sampled particles.  Every loop returns
 * the number of pair interactions it evaluated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

typedef struct {
    double gamma;         /* adiabatic index */
    double kernel_gamma;  /* H = kernel_gamma * h */
    double beta_visc;     /* signal-velocity factor on the approach speed */
    double balsara_eps;   /* regulariser of the Balsara switch, times c/h */
    double support_eps;   /* neighbour test uses r^2 < H^2 (1 + support_eps);
                             only shifts max-type outputs and pair counts,
                             since W and dW/dr vanish at r >= H */
    double box[3];        /* periodic box edges */
    int32_t active_bin;   /* force loop: particle i active iff time_bin <= it */
    int32_t pad;
} oracle_params;

/* ------------------------------------------------------------------------ */
/* Kernel: W(r, H) = (8/pi) / H^3 * w(r/H)                                   */
/*   w(q) = 1 - 6 q^2 + 6 q^3      0 <= q < 1/2                              */
/*        = 2 (1 - q)^3            1/2 <= q < 1                              */
/*        = 0                      q >= 1                                    */
/* ------------------------------------------------------------------------ */
static const double KERNEL_NORM = 8.0 / ORACLE_PI;

double oracle_w(double q)
{
    if (q < 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;
    if (q < 1.0) return 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
    return 0.0;
}

double oracle_dw(double q) /* dw/dq */
{
    if (q < 0.5) return -12.0 * q + 18.0 * q * q;
    if (q < 1.0) return -6.0 * (1.0 - q) * (1.0 - q);
    return 0.0;
}

double oracle_W(double r, double H)
{
    return KERNEL_NORM / (H * H * H) * oracle_w(r / H);
}

double oracle_dWdr(double r, double H)
{
    return KERNEL_NORM / (H * H * H * H) * oracle_dw(r / H);
}

double oracle_dWdH(double r, double H)
{
    double q = r / H;
    return -KERNEL_NORM / (H * H * H * H) * (3.0 * oracle_w(q) + q * oracle_dw(q));
}

/* Minimum-image separation x_i - x_j in a periodic box. */
static void min_image(const double *xi, const double *xj, const double *box,
                      double *d)
{
    for (int k = 0; k < 3; ++k) {
        double s = xi[k] - xj[k];
        s -= box[k] * nearbyint(s / box[k]);
        d[k] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Density loop (Sec. 2.1, Table 1 p-d / u-d).  Raw sums over j != i with    */
/* r_ij < H_i; the self contribution and the 1/rho of div/rot are the        */
/* ghost's job.                                                              */
/*   out[8 k + 0] = sum m_j W(r, H_i)                       (rho)            */
/*   out[8 k + 1] = sum m_j dW/dH(r, H_i)                   (d rho / d H)    */
/*   out[8 k + 2] = sum (4 pi / 3) H_i^3 W(r, H_i)          (wcount)         */
/*   out[8 k + 3] = d/dH_i of the wcount sum (the H^3 factor included)       */
/*   out[8 k + 4] = -sum m_j v_ij . rhat F_i                (rho div v)      */
/*   out[8 k + 5..7] = sum m_j v_ij x rhat F_i              (rho curl v)     */
/* with v_ij = v_i - v_j, rhat = (x_i - x_j) / r, F_i = dW/dr(r, H_i).       */
/* ------------------------------------------------------------------------ */
int64_t oracle_density(int64_t n, const double *x, const float *v,
                       const float *m, const float *h, const oracle_params *P,
                       int64_t nsel, const int64_t *sel, double *out)
{
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : pairs)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        double Hi = P->kernel_gamma * (double)h[i];
        double H2 = Hi * Hi * (1.0 + P->support_eps);
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], P->box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < H2)) continue;
            pairs++;
            double r = sqrt(r2);
            double mj = (double)m[j];
            double F = oracle_dWdr(r, Hi);
            double rh[3] = {0, 0, 0};
            if (r > 0.0) { rh[0] = d[0] / r; rh[1] = d[1] / r; rh[2] = d[2] / r; }
            double vij[3];
            for (int c = 0; c < 3; ++c) vij[c] = (double)v[3 * i + c] - (double)v[3 * j + c];
            acc[0] += mj * oracle_W(r, Hi);
            acc[1] += mj * oracle_dWdH(r, Hi);
            acc[2] += (4.0 * ORACLE_PI / 3.0) * Hi * Hi * Hi * oracle_W(r, Hi);
            /* d/dH [ (4pi/3) H^3 W(r,H) ] = (4pi/3) (3 H^2 W + H^3 dW/dH) */
            acc[3] += (4.0 * ORACLE_PI / 3.0) *
                      (3.0 * Hi * Hi * oracle_W(r, Hi) + Hi * Hi * Hi * oracle_dWdH(r, Hi));
            acc[4] += -mj * (vij[0] * rh[0] + vij[1] * rh[1] + vij[2] * rh[2]) * F;
            acc[5] += mj * (vij[1] * rh[2] - vij[2] * rh[1]) * F;
            acc[6] += mj * (vij[2] * rh[0] - vij[0] * rh[2]) * F;
            acc[7] += mj * (vij[0] * rh[1] - vij[1] * rh[0]) * F;
        }
        for (int c = 0; c < 8; ++c) out[8 * k + c] = acc[c];
    }
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Conditioning scales of the two h-derivative sums of the density loop.     */
/* Their terms change sign at q = 1/2 and largely cancel, so the value says  */
/* nothing about the rounding a sum of them can carry; the sum of the terms' */
/* magnitudes does.  The self term of wcount_dh is an exact cancellation,   */
/* (4 pi / 3)(3 H^2 W(0) + H^3 dW/dH(0)) = 0, which any evaluation leaves as */
/* a rounding residue of its parts, so it enters with the magnitude of its   */
/* two parts.  These are tolerance scales for comparisons, not results of   */
/* the method.                                                               */
/*   out[2 k + 0] = m_i |dW/dH(0, H_i)| + sum m_j |dW/dH(r, H_i)|            */
/*   out[2 k + 1] = (4 pi / 3)(3 H^2 W(0) + H^3 |dW/dH(0)|)                  */
/*                  + sum (4 pi / 3) |3 H^2 W + H^3 dW/dH|                   */
/* over j != i with r_ij < H_i.                                              */
/* ------------------------------------------------------------------------ */
void oracle_dh_scales(int64_t n, const double *x, const float *m, const float *h,
                      const oracle_params *P, int64_t nsel, const int64_t *sel,
                      double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        double Hi = P->kernel_gamma * (double)h[i];
        double H2 = Hi * Hi * (1.0 + P->support_eps);
        double c = 4.0 * ORACLE_PI / 3.0;
        double s_rho = (double)m[i] * fabs(oracle_dWdH(0.0, Hi));
        double s_w = c * (3.0 * Hi * Hi * oracle_W(0.0, Hi) +
                          Hi * Hi * Hi * fabs(oracle_dWdH(0.0, Hi)));
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], P->box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < H2)) continue;
            double r = sqrt(r2);
            s_rho += (double)m[j] * fabs(oracle_dWdH(r, Hi));
            s_w += c * fabs(3.0 * Hi * Hi * oracle_W(r, Hi) + Hi * Hi * Hi * oracle_dWdH(r, Hi));
        }
        out[2 * k + 0] = s_rho;
        out[2 * k + 1] = s_w;
    }
}

/* ------------------------------------------------------------------------ */
/* Ghost after density (the linear update of Sec. 2.1).                      */
/*   rho += m_i W(0, H_i); rho_dh += m_i dW/dH(0, H_i); wcount += its self   */
/*   term; div v = raw / rho; curl v = raw / rho;                            */
/*   Omega = 1 + H/(3 rho) d rho/dH;  f_gradh = 1/Omega, except for a       */
/*   particle with no neighbour inside its support (raw wcount sum 0), whose */
/*   Omega is exactly 0: f_gradh = 1 (no grad-h correction).                 */
/*   P = (gamma - 1) rho u;  c = sqrt(gamma (gamma - 1) u);                  */
/*   Balsara B = |div v| / (|div v| + |curl v| + eps c / h).                 */
/* out[12 k + ...] = rho, rho_dh, wcount, wcount_dh, div_v, rot_v[3],        */
/*                   f_gradh, P, c, B                                        */
/* ------------------------------------------------------------------------ */
void oracle_ghost(int64_t nsel, const int64_t *sel, const float *m,
                  const float *h, const float *u, const double *dens,
                  const oracle_params *P, double *out)
{
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        double Hi = P->kernel_gamma * (double)h[i];
        double mi = (double)m[i];
        const double *s = &dens[8 * k];
        double rho = s[0] + mi * oracle_W(0.0, Hi);
        double rho_dh = s[1] + mi * oracle_dWdH(0.0, Hi);
        double wcount = s[2] + (4.0 * ORACLE_PI / 3.0) * Hi * Hi * Hi * oracle_W(0.0, Hi);
        double wcount_dh = s[3] + (4.0 * ORACLE_PI / 3.0) *
                                  (3.0 * Hi * Hi * oracle_W(0.0, Hi) +
                                   Hi * Hi * Hi * oracle_dWdH(0.0, Hi));
        double div = s[4] / rho;
        double rot[3] = {s[5] / rho, s[6] / rho, s[7] / rho};
        double omega = 1.0 + Hi / (3.0 * rho) * rho_dh;
        double fgh = s[2] == 0.0 ? 1.0 : 1.0 / omega;
        double ui = (double)u[i];
        double pres = (P->gamma - 1.0) * rho * ui;
        double cs = sqrt(P->gamma * (P->gamma - 1.0) * ui);
        double arot = sqrt(rot[0] * rot[0] + rot[1] * rot[1] + rot[2] * rot[2]);
        double bal = fabs(div) / (fabs(div) + arot + P->balsara_eps * cs / (double)h[i]);
        double *o = &out[12 * k];
        o[0] = rho; o[1] = rho_dh; o[2] = wcount; o[3] = wcount_dh;
        o[4] = div; o[5] = rot[0]; o[6] = rot[1]; o[7] = rot[2];
        o[8] = fgh; o[9] = pres; o[10] = cs; o[11] = bal;
    }
}

/* ------------------------------------------------------------------------ */
/* Gradient loop (Sec. 2.1, Table 1 p-g), over j with r < H_i:               */
/*   v_sig_grad_i = max_j (c_i + c_j - beta min(0, v_ij . rhat))  (init 0)   */
/*   laplace_u_i  = sum_j 2 m_j (u_i - u_j) / rho_j * F_i / r                */
/* with c = sqrt(gamma (gamma - 1) u).  out[2 k + ...]                        */
/* ------------------------------------------------------------------------ */
int64_t oracle_gradient(int64_t n, const double *x, const float *v,
                        const float *m, const float *h, const float *u,
                        const double *rho, const oracle_params *P,
                        int64_t nsel, const int64_t *sel, double *out)
{
    int64_t pairs = 0;
    double gg = P->gamma * (P->gamma - 1.0);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : pairs)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        double Hi = P->kernel_gamma * (double)h[i];
        double H2 = Hi * Hi * (1.0 + P->support_eps);
        double ci = sqrt(gg * (double)u[i]);
        double vsig = 0.0, lap = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], P->box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < H2)) continue;
            pairs++;
            double r = sqrt(r2);
            double rh[3] = {0, 0, 0};
            if (r > 0.0) { rh[0] = d[0] / r; rh[1] = d[1] / r; rh[2] = d[2] / r; }
            double w = 0.0;
            for (int c = 0; c < 3; ++c)
                w += ((double)v[3 * i + c] - (double)v[3 * j + c]) * rh[c];
            double cj = sqrt(gg * (double)u[j]);
            double vs = ci + cj - P->beta_visc * fmin(0.0, w);
            if (vs > vsig) vsig = vs;
            if (r > 0.0)
                lap += 2.0 * (double)m[j] * ((double)u[i] - (double)u[j]) / rho[j] *
                       oracle_dWdr(r, Hi) / r;
        }
        out[2 * k + 0] = vsig;
        out[2 * k + 1] = lap;
    }
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Force loop (Sec. 2.1, Table 1 p-f / u-f), over j with r < max(H_i, H_j). */
/*   F_i = dW/dr(r, H_i), F_j = dW/dr(r, H_j), Fbar = (F_i + F_j)/2          */
/*   w = v_ij . rhat, mu = min(0, w), rhobar = (rho_i + rho_j)/2             */
/*   alpha_ij = (alpha_i B_i + alpha_j B_j)/2, vsig_ij = c_i + c_j - beta mu */
/*   Pi_ij = -alpha_ij vsig_ij mu / rhobar                                   */
/*   a_i    = -sum m_j [f_i P_i/rho_i^2 F_i + f_j P_j/rho_j^2 F_j            */
/*                      + Pi_ij Fbar] rhat                                   */
/*   du_i/dt = sum m_j [f_i P_i/rho_i^2 F_i w + 1/2 Pi_ij Fbar w             */
/*             + alphaD_ij sqrt(|P_i - P_j|/rhobar) (u_i - u_j) Fbar/rhobar] */
/*   dh_i/dt = -(h_i/3) f_i / rho_i sum m_j w F_i                            */
/*   v_sig_i = max_j vsig_ij  (init 0)                                        */
/* Particles with time_bin > active_bin are not updated (outputs 0, flag 0). */
/* out[6 k + ...] = a[3], u_dt, h_dt, v_sig                                   */
/* ------------------------------------------------------------------------ */
int64_t oracle_force(int64_t n, const double *x, const float *v, const float *m,
                     const float *h, const float *u, const double *rho,
                     const double *fgh, const double *pres, const double *cs,
                     const double *bal, const float *alpha_v,
                     const float *alpha_d, const int8_t *tbin,
                     const oracle_params *P, int64_t nsel, const int64_t *sel,
                     double *out)
{
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : pairs)
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t i = sel ? sel[k] : k;
        double *o = &out[6 * k];
        for (int c = 0; c < 6; ++c) o[c] = 0.0;
        if ((int32_t)tbin[i] > P->active_bin) continue;
        double Hi = P->kernel_gamma * (double)h[i];
        double Ai = fgh[i] * pres[i] / (rho[i] * rho[i]);
        double acc[3] = {0, 0, 0}, udt = 0.0, hsum = 0.0, vsig = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double Hj = P->kernel_gamma * (double)h[j];
            double Hm = Hi > Hj ? Hi : Hj;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], P->box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < Hm * Hm * (1.0 + P->support_eps))) continue;
            pairs++;
            double r = sqrt(r2);
            double rh[3] = {0, 0, 0};
            if (r > 0.0) { rh[0] = d[0] / r; rh[1] = d[1] / r; rh[2] = d[2] / r; }
            double w = 0.0;
            for (int c = 0; c < 3; ++c)
                w += ((double)v[3 * i + c] - (double)v[3 * j + c]) * rh[c];
            double mu = fmin(0.0, w);
            double Fi = oracle_dWdr(r, Hi);
            double Fj = oracle_dWdr(r, Hj);
            double Fbar = 0.5 * (Fi + Fj);
            double rhobar = 0.5 * (rho[i] + rho[j]);
            double alpha = 0.5 * ((double)alpha_v[i] * bal[i] + (double)alpha_v[j] * bal[j]);
            double vs = cs[i] + cs[j] - P->beta_visc * mu;
            double Pi = -alpha * vs * mu / rhobar;
            double Aj = fgh[j] * pres[j] / (rho[j] * rho[j]);
            double mj = (double)m[j];
            double s = Ai * Fi + Aj * Fj + Pi * Fbar;
            for (int c = 0; c < 3; ++c) acc[c] -= mj * s * rh[c];
            double alphaD = 0.5 * ((double)alpha_d[i] + (double)alpha_d[j]);
            double cond = alphaD * sqrt(fabs(pres[i] - pres[j]) / rhobar) *
                          ((double)u[i] - (double)u[j]) * Fbar / rhobar;
            udt += mj * (Ai * Fi * w + 0.5 * Pi * Fbar * w + cond);
            hsum += mj * w * Fi;
            if (vs > vsig) vsig = vs;
        }
        o[0] = acc[0]; o[1] = acc[1]; o[2] = acc[2];
        o[3] = udt;
        o[4] = -((double)h[i] / 3.0) * fgh[i] / rho[i] * hsum;
        o[5] = vsig;
    }
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Cell grid (Sec. 2.2).  Octree rule for a uniform particle set: halve the  */
/* box edge while the half is still >= H_max = kernel_gamma * max h, so the  */
/* leaf edge lies in [H_max, 2 H_max) and every neighbour of a particle is in */
/* its own or an adjacent cell.  ncell_in[d] > 0 overrides the count (it must */
/* still give edges >= H_max).  At least 3 cells per dimension are required  */
/* so that periodic pair tasks are unique.  Particle cell index:             */
/* c = ix + nx (iy + ny iz), ix = floor(x / box * nx) clamped.  Particles are */
/* sorted by cell with a stable counting sort: perm[k] = original index of   */
/* the k-th particle in cell order.                                          */
/* Returns 0, or -1 if the grid is invalid.                                  */
/* ------------------------------------------------------------------------ */
int oracle_grid(int64_t n, const double *x, const float *h, const double *box,
                double kernel_gamma, const int32_t *ncell_in, int32_t *ncell_out,
                int64_t *perm, int64_t *cell_start)
{
    double hmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if ((double)h[i] > hmax) hmax = (double)h[i];
    double Hmax = kernel_gamma * hmax;
    int32_t nc[3];
    for (int d = 0; d < 3; ++d) {
        if (ncell_in && ncell_in[d] > 0) {
            nc[d] = ncell_in[d];
            if (box[d] / nc[d] < Hmax) return -1;
        } else {
            int32_t k = 1;
            while (box[d] / (2.0 * k) >= Hmax && k < (1 << 20)) k *= 2;
            nc[d] = k;
        }
        if (nc[d] < 3) return -1;
        ncell_out[d] = nc[d];
    }
    if (!perm || !cell_start) return 0;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t idx[3];
        for (int d = 0; d < 3; ++d) {
            int64_t k = (int64_t)floor(x[3 * i + d] / box[d] * nc[d]);
            if (k < 0) k = 0;
            if (k >= nc[d]) k = nc[d] - 1;
            idx[d] = k;
        }
        cell[i] = idx[0] + nc[0] * (idx[1] + nc[1] * idx[2]);
        cell_start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    for (int64_t c = 0; c < ncell; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Task list (Sec. 2.2-2.3).  For each cell c in increasing index: a self     */
/* task (c, -1) if c is not empty, then one pair task (c, c') for each of the */
/* 13 neighbour offsets that come after (0,0,0) when (dz, dy, dx) run over    */
/* {-1,0,1}^3 with dz outermost and dx innermost, c' = c + offset wrapped     */
/* periodically, skipped if either cell is empty.  shift[3 t + d] is -1, 0 or */
/* +1: the particles of c' are moved by shift * box so that they sit next to */
/* c (the periodic shift applied at pack time).  Returns the task count;      */
/* the arrays may be NULL to count only.                                      */
/* ------------------------------------------------------------------------ */
int64_t oracle_tasks(const int32_t *nc, const int64_t *cell_start, int32_t *ci,
                     int32_t *cj, int8_t *shift)
{
    int64_t nt = 0;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t cnt = cell_start[c + 1] - cell_start[c];
        if (cnt == 0) continue;
        if (ci) { ci[nt] = (int32_t)c; cj[nt] = -1; shift[3 * nt] = shift[3 * nt + 1] = shift[3 * nt + 2] = 0; }
        nt++;
        int64_t ix = c % nc[0], iy = (c / nc[0]) % nc[1], iz = c / ((int64_t)nc[0] * nc[1]);
        int seen_center = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0 && dz == 0) { seen_center = 1; continue; }
                    if (!seen_center) continue;
                    int64_t p[3] = {ix + dx, iy + dy, iz + dz};
                    int8_t s[3];
                    for (int d = 0; d < 3; ++d) {
                        s[d] = 0;
                        if (p[d] < 0) { p[d] += nc[d]; s[d] = -1; }
                        else if (p[d] >= nc[d]) { p[d] -= nc[d]; s[d] = 1; }
                    }
                    int64_t c2 = p[0] + nc[0] * (p[1] + nc[1] * p[2]);
                    if (cell_start[c2 + 1] - cell_start[c2] == 0) continue;
                    if (ci) {
                        ci[nt] = (int32_t)c; cj[nt] = (int32_t)c2;
                        shift[3 * nt] = s[0]; shift[3 * nt + 1] = s[1]; shift[3 * nt + 2] = s[2];
                    }
                    nt++;
                }
    }
    return nt;
}

static int64_t cell_count(const int64_t *cell_start, int32_t c)
{
    return c < 0 ? 0 : cell_start[c + 1] - cell_start[c];
}

/* Bundles (Sec. 2.3): consecutive task ranges; a bundle takes tasks while its */
/* slot total stays <= max_slots (always at least one task; max_slots <= 0    */
/* puts every task in one bundle).  A self task has |c| slots, a pair task    */
/* |ci| + |cj|.  bundle_start has nb + 1 entries; returns nb.                 */
int64_t oracle_bundles(int64_t ntasks, const int32_t *ci, const int32_t *cj,
                       const int64_t *cell_start, int64_t max_slots,
                       int64_t *bundle_start)
{
    int64_t nb = 0, slots = 0;
    if (bundle_start) bundle_start[0] = 0;
    for (int64_t t = 0; t < ntasks; ++t) {
        int64_t s = cell_count(cell_start, ci[t]) + cell_count(cell_start, cj[t]);
        if (t > 0 && max_slots > 0 && slots + s > max_slots) {
            nb++;
            if (bundle_start) bundle_start[nb] = t;
            slots = 0;
        }
        slots += s;
    }
    if (ntasks > 0) nb++;
    if (bundle_start) bundle_start[nb] = ntasks;
    return nb;
}

/* ------------------------------------------------------------------------ */
/* Logical fields, original particle order (the Table 1 catalogue plus the   */
/* Sphenix quantities the loops need).  NULL = not present.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *x; float *v; float *a; float *mass; float *h; float *u;
    float *u_dt; float *rho; int8_t *time_bin; float *alpha_visc;
    float *alpha_diff; float *rho_dh; float *wcount; float *wcount_dh;
    float *div_v; float *rot_v; float *f_gradh; float *pressure;
    float *soundspeed; float *balsara; float *v_sig_grad; float *laplace_u;
    float *h_dt; float *v_sig; int64_t *id;
} oracle_fields;

/* ------------------------------------------------------------------------ */
/* Packed buffers.  A bundle of S slots is a sequence of lanes; lane k holds  */
/* S elements of its size and starts at sum_{l<k} round_up(S * size_l, 256).  */
/* Slots of a task are contiguous: ci's particles then cj's, each in cell     */
/* order; tasks follow in bundle order.                                       */
/*  density  in : x0 x1 x2 (f64) | {vx vy vz m} (4 x f32) | h                 */
/*  gradient in : density in | u | rho                                        */
/*  force    in : gradient in | f_gradh | balsara | alpha_visc | alpha_diff | */
/*                time_bin (i8)                                               */
/*  density  out: {rho rho_dh wcount wcount_dh} | {div_v rot_x rot_y rot_z}   */
/*  gradient out: {v_sig_grad laplace_u}                                      */
/*  force    out: {ax ay az u_dt} | {h_dt v_sig}                              */
/* ------------------------------------------------------------------------ */
enum { O_DENSITY = 0, O_GRADIENT = 1, O_FORCE = 2 };

static int64_t round256(int64_t b) { return (b + 255) / 256 * 256; }

static int lanes_in(int loop, int64_t *sz)
{
    int k = 0;
    sz[k++] = 8; sz[k++] = 8; sz[k++] = 8; sz[k++] = 16; sz[k++] = 4;
    if (loop >= O_GRADIENT) { sz[k++] = 4; sz[k++] = 4; }
    if (loop == O_FORCE) { sz[k++] = 4; sz[k++] = 4; sz[k++] = 4; sz[k++] = 4; sz[k++] = 1; }
    return k;
}

static int lanes_out(int loop, int64_t *sz)
{
    if (loop == O_DENSITY) { sz[0] = 16; sz[1] = 16; return 2; }
    if (loop == O_GRADIENT) { sz[0] = 8; return 1; }
    sz[0] = 16; sz[1] = 8; return 2;
}

static int64_t lane_offsets(int nl, const int64_t *sz, int64_t S, int64_t *off)
{
    int64_t o = 0;
    for (int k = 0; k < nl; ++k) { off[k] = o; o += round256(S * sz[k]); }
    return o;
}

static int64_t bundle_slots(int64_t t0, int64_t t1, const int32_t *ci,
                            const int32_t *cj, const int64_t *cell_start)
{
    int64_t s = 0;
    for (int64_t t = t0; t < t1; ++t)
        s += cell_count(cell_start, ci[t]) + cell_count(cell_start, cj[t]);
    return s;
}

int64_t oracle_buffer_bytes(int loop, int in_or_out, int64_t nslots)
{
    int64_t sz[16], off[16];
    int nl = in_or_out == 0 ? lanes_in(loop, sz) : lanes_out(loop, sz);
    return lane_offsets(nl, sz, nslots, off);
}

/* Pack the view of `loop` for tasks [t0, t1) into buf.  x of the cj side is  */
/* x + shift * box in FP64 (one rounding); every other value is copied.       */
int oracle_pack(int loop, const oracle_fields *f, const int64_t *perm,
                const int64_t *cell_start, const int32_t *ci, const int32_t *cj,
                const int8_t *shift, int64_t t0, int64_t t1, const double *box,
                uint8_t *buf)
{
    int64_t sz[16], off[16];
    int nl = lanes_in(loop, sz);
    int64_t S = bundle_slots(t0, t1, ci, cj, cell_start);
    lane_offsets(nl, sz, S, off);
    int64_t slot = 0;
    for (int64_t t = t0; t < t1; ++t) {
        for (int side = 0; side < 2; ++side) {
            int32_t c = side == 0 ? ci[t] : cj[t];
            if (c < 0) continue;
            for (int64_t k = cell_start[c]; k < cell_start[c + 1]; ++k, ++slot) {
                int64_t p = perm[k];
                for (int d = 0; d < 3; ++d) {
                    double xv = f->x[3 * p + d];
                    if (side == 1 && shift[3 * t + d] != 0)
                        xv = xv + (double)shift[3 * t + d] * box[d];
                    memcpy(buf + off[d] + 8 * slot, &xv, 8);
                }
                float vm[4] = {f->v[3 * p], f->v[3 * p + 1], f->v[3 * p + 2], f->mass[p]};
                memcpy(buf + off[3] + 16 * slot, vm, 16);
                memcpy(buf + off[4] + 4 * slot, &f->h[p], 4);
                if (loop >= O_GRADIENT) {
                    memcpy(buf + off[5] + 4 * slot, &f->u[p], 4);
                    memcpy(buf + off[6] + 4 * slot, &f->rho[p], 4);
                }
                if (loop == O_FORCE) {
                    memcpy(buf + off[7] + 4 * slot, &f->f_gradh[p], 4);
                    memcpy(buf + off[8] + 4 * slot, &f->balsara[p], 4);
                    memcpy(buf + off[9] + 4 * slot, &f->alpha_visc[p], 4);
                    memcpy(buf + off[10] + 4 * slot, &f->alpha_diff[p], 4);
                    memcpy(buf + off[11] + 1 * slot, &f->time_bin[p], 1);
                }
            }
        }
    }
    return 0;
}

/* Unpack (Sec. 2.3): for every particle touched by tasks [t0, t1), fold its */
/* slots in increasing task order (ci before cj) into its fields.  Sums use  */
/* Kahan's compensated summation in FP32, starting from the stored value     */
/* with zero compensation (y = x - c; t = s + y; c = (t - s) - y; s = t);     */
/* the signal velocities take the max (fmaxf).                               */
typedef struct {
    int lane;      /* output lane */
    int col;       /* float index inside the lane element */
    float *field;  /* destination logical field */
    int ncomp;     /* components per particle of that field */
    int comp;      /* component written */
    int is_max;    /* 1: max reduction, 0: compensated sum */
} unpack_col;

static int unpack_columns(int loop, oracle_fields *f, unpack_col *c)
{
    if (loop == O_DENSITY) {
        unpack_col t[8] = {{0, 0, f->rho, 1, 0, 0}, {0, 1, f->rho_dh, 1, 0, 0},
                           {0, 2, f->wcount, 1, 0, 0}, {0, 3, f->wcount_dh, 1, 0, 0},
                           {1, 0, f->div_v, 1, 0, 0}, {1, 1, f->rot_v, 3, 0, 0},
                           {1, 2, f->rot_v, 3, 1, 0}, {1, 3, f->rot_v, 3, 2, 0}};
        memcpy(c, t, sizeof(t));
        return 8;
    }
    if (loop == O_GRADIENT) {
        unpack_col t[2] = {{0, 0, f->v_sig_grad, 1, 0, 1}, {0, 1, f->laplace_u, 1, 0, 0}};
        memcpy(c, t, sizeof(t));
        return 2;
    }
    unpack_col t[6] = {{0, 0, f->a, 3, 0, 0}, {0, 1, f->a, 3, 1, 0}, {0, 2, f->a, 3, 2, 0},
                       {0, 3, f->u_dt, 1, 0, 0}, {1, 0, f->h_dt, 1, 0, 0},
                       {1, 1, f->v_sig, 1, 0, 1}};
    memcpy(c, t, sizeof(t));
    return 6;
}

int oracle_unpack(int loop, oracle_fields *f, int64_t n, const int64_t *perm,
                  const int64_t *cell_start, const int32_t *ci, const int32_t *cj,
                  int64_t t0, int64_t t1, const uint8_t *buf)
{
    int64_t sz[16], off[16];
    int nl = lanes_out(loop, sz);
    int64_t S = bundle_slots(t0, t1, ci, cj, cell_start);
    lane_offsets(nl, sz, S, off);
    unpack_col col[8];
    int ncol = unpack_columns(loop, f, col);
    /* per particle and column: running sum s and compensation c */
    float *sum = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * 8);
    float *cmp = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * 8);
    uint8_t *touched = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t slot = 0;
    for (int64_t t = t0; t < t1; ++t) {
        for (int side = 0; side < 2; ++side) {
            int32_t c = side == 0 ? ci[t] : cj[t];
            if (c < 0) continue;
            for (int64_t k = cell_start[c]; k < cell_start[c + 1]; ++k, ++slot) {
                int64_t p = perm[k];
                if (!touched[p]) {
                    touched[p] = 1;
                    for (int q = 0; q < ncol; ++q) {
                        sum[8 * p + q] = col[q].field[col[q].ncomp * p + col[q].comp];
                        cmp[8 * p + q] = 0.0f;
                    }
                }
                for (int q = 0; q < ncol; ++q) {
                    float val;
                    memcpy(&val, buf + off[col[q].lane] + sz[col[q].lane] * slot + 4 * col[q].col, 4);
                    if (col[q].is_max) {
                        float *d = &col[q].field[col[q].ncomp * p + col[q].comp];
                        *d = fmaxf(*d, val);
                    } else {
                        volatile float y = val - cmp[8 * p + q];
                        volatile float tsum = sum[8 * p + q] + y;
                        cmp[8 * p + q] = (tsum - sum[8 * p + q]) - y;
                        sum[8 * p + q] = tsum;
                    }
                }
            }
        }
    }
    for (int64_t p = 0; p < n; ++p) {
        if (!touched[p]) continue;
        for (int q = 0; q < ncol; ++q)
            if (!col[q].is_max)
                col[q].field[col[q].ncomp * p + col[q].comp] = sum[8 * p + q];
    }
    free(sum);
    free(cmp);
    free(touched);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Store layouts (Sec. 3.1).  A layout is a sequence of substructs; each is  */
/* a C struct of its members with natural alignment (member offset rounded   */
/* up to the member's element size, struct size rounded up to the largest    */
/* element size).  Substruct arrays follow each other in memory, each        */
/* starting on a 256-byte boundary.  Unused bytes are zero.                  */
/* ------------------------------------------------------------------------ */
enum {
    F_X, F_V, F_A, F_MASS, F_H, F_U, F_UDT, F_RHO, F_TBIN, F_AVISC, F_ADIFF,
    F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV, F_ROTV, F_FGRADH, F_PRES, F_CS,
    F_BALS, F_VSIGG, F_LAPU, F_HDT, F_VSIG, F_ID, F_BALLAST, F_NUM
};
/* element size, number of elements, type class (0 double, 1 float, 2 int) */
static const int FIELD_ELEM[F_NUM] = {8, 4, 4, 4, 4, 4, 4, 4, 1, 4, 4, 4, 4, 4,
                                      4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 8, 1};
static const int FIELD_COUNT[F_NUM] = {3, 3, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                       1, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 8};
static const int FIELD_CLASS[F_NUM] = {0, 1, 1, 1, 1, 1, 1, 1, 2, 1, 1, 1, 1, 1,
                                       1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2};

enum {
    L_AOS, L_AOS_RANDOM, L_PACK_GRAD, L_PACK_FORCE, L_PACK_SHARED,
    L_PACK_GRAD_TYPE, L_PACK_FORCE_TYPE, L_PACK_SHARED_TYPE, L_SOA,
    L_PACK_FORCE_REPL, L_FUSED, L_NUM
};

#define MAXG 64
typedef struct {
    int ngroups;
    int nmem[MAXG];
    int field[MAXG][F_NUM];
    int comp[MAXG][F_NUM];   /* SoA: the single component, else -1 (all) */
} layout_def;

/* SplitMix64 (Steele, Lea & Flood 2014; Vigna's public-domain statement):   */
/* state += 0x9E3779B97F4A7C15; z = state; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; */
/* z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31.                   */
uint64_t oracle_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void add_group(layout_def *L, const int *fields, int nf)
{
    int g = L->ngroups++;
    L->nmem[g] = nf;
    for (int k = 0; k < nf; ++k) { L->field[g][k] = fields[k]; L->comp[g][k] = -1; }
}

/* Split a group by type class: double members, then float, then int. */
static void add_group_typed(layout_def *L, const int *fields, int nf, int by_type)
{
    if (!by_type) { add_group(L, fields, nf); return; }
    for (int cls = 0; cls < 3; ++cls) {
        int sub[F_NUM], ns = 0;
        for (int k = 0; k < nf; ++k)
            if (FIELD_CLASS[fields[k]] == cls) sub[ns++] = fields[k];
        if (ns) add_group(L, sub, ns);
    }
}

static int build_layout(int layout, uint64_t seed, layout_def *L)
{
    /* use order: Table 1 rows first, then the remaining members */
    static const int aos[F_NUM] = {F_X, F_V, F_A, F_MASS, F_H, F_U, F_UDT, F_RHO,
        F_TBIN, F_AVISC, F_ADIFF, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV, F_ROTV,
        F_FGRADH, F_PRES, F_CS, F_BALS, F_VSIGG, F_LAPU, F_HDT, F_VSIG, F_ID,
        F_BALLAST};
    static const int grad_view[] = {F_X, F_V, F_MASS, F_H, F_U, F_RHO};
    static const int force_only[] = {F_TBIN, F_FGRADH, F_BALS, F_AVISC, F_ADIFF};
    static const int force_view[] = {F_X, F_V, F_MASS, F_H, F_U, F_RHO, F_TBIN,
                                     F_FGRADH, F_BALS, F_AVISC, F_ADIFF};
    static const int shared3[] = {F_X, F_V, F_MASS, F_H};
    static const int u_rho[] = {F_U, F_RHO};
    static const int dens_out[] = {F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV, F_ROTV};
    static const int grad_out[] = {F_VSIGG, F_LAPU};
    static const int force_out[] = {F_A, F_UDT, F_HDT, F_VSIG};
    static const int rest[] = {F_PRES, F_CS, F_ID, F_BALLAST};
    /* replication (Sec. 5, outlook): the density view's inputs stored again */
    static const int dens_view[] = {F_X, F_V, F_MASS, F_H};
    /* fused views: each loop's inputs with the outputs its unpack writes */
    static const int fused_dens[] = {F_X, F_V, F_MASS, F_H, F_RHO, F_RHODH, F_WCOUNT,
                                     F_WCOUNTDH, F_DIVV, F_ROTV};
    static const int fused_grad[] = {F_U, F_VSIGG, F_LAPU};
    static const int fused_force[] = {F_TBIN, F_FGRADH, F_BALS, F_AVISC, F_ADIFF, F_A,
                                      F_UDT, F_HDT, F_VSIG};
    memset(L, 0, sizeof(*L));
    int by_type = layout == L_PACK_GRAD_TYPE || layout == L_PACK_FORCE_TYPE ||
                  layout == L_PACK_SHARED_TYPE;
    switch (layout) {
    case L_AOS:
        add_group(L, aos, F_NUM);
        break;
    case L_AOS_RANDOM: {
        int order[F_NUM];
        memcpy(order, aos, sizeof(order));
        uint64_t st = seed;
        for (int i = F_NUM - 1; i > 0; --i) {
            int j = (int)(oracle_splitmix64(&st) % (uint64_t)(i + 1));
            int tmp = order[i]; order[i] = order[j]; order[j] = tmp;
        }
        add_group(L, order, F_NUM);
        break;
    }
    case L_PACK_GRAD: case L_PACK_GRAD_TYPE:
        add_group_typed(L, grad_view, 6, by_type);
        add_group_typed(L, force_only, 5, by_type);
        add_group_typed(L, dens_out, 5, by_type);
        add_group_typed(L, grad_out, 2, by_type);
        add_group_typed(L, force_out, 4, by_type);
        add_group_typed(L, rest, 4, by_type);
        break;
    case L_PACK_FORCE: case L_PACK_FORCE_TYPE:
        add_group_typed(L, force_view, 11, by_type);
        add_group_typed(L, dens_out, 5, by_type);
        add_group_typed(L, grad_out, 2, by_type);
        add_group_typed(L, force_out, 4, by_type);
        add_group_typed(L, rest, 4, by_type);
        break;
    case L_PACK_SHARED: case L_PACK_SHARED_TYPE:
        add_group_typed(L, shared3, 4, by_type);
        add_group_typed(L, u_rho, 2, by_type);
        add_group_typed(L, force_only, 5, by_type);
        add_group_typed(L, dens_out, 5, by_type);
        add_group_typed(L, grad_out, 2, by_type);
        add_group_typed(L, force_out, 4, by_type);
        add_group_typed(L, rest, 4, by_type);
        break;
    case L_PACK_FORCE_REPL:
        add_group(L, dens_view, 4);
        add_group(L, force_view, 11);
        add_group(L, dens_out, 5);
        add_group(L, grad_out, 2);
        add_group(L, force_out, 4);
        add_group(L, rest, 4);
        break;
    case L_FUSED:
        add_group(L, fused_dens, 10);
        add_group(L, fused_grad, 3);
        add_group(L, fused_force, 9);
        add_group(L, rest, 4);
        break;
    case L_SOA:
        for (int k = 0; k < F_NUM; ++k) {
            int f = aos[k];
            if (f == F_BALLAST) {        /* opaque bytes: one array */
                add_group(L, &f, 1);
                continue;
            }
            for (int c = 0; c < FIELD_COUNT[f]; ++c) {
                int g = L->ngroups++;
                L->nmem[g] = 1; L->field[g][0] = f; L->comp[g][0] = FIELD_COUNT[f] > 1 ? c : -1;
            }
        }
        break;
    default:
        return -1;
    }
    return 0;
}

/* member bytes: a whole field, or one component of it in SoA */
static int member_bytes(const layout_def *L, int g, int k)
{
    int f = L->field[g][k];
    return L->comp[g][k] >= 0 ? FIELD_ELEM[f] : FIELD_ELEM[f] * FIELD_COUNT[f];
}

static int group_record(const layout_def *L, int g, int *offs)
{
    int o = 0, al = 1;
    for (int k = 0; k < L->nmem[g]; ++k) {
        int e = FIELD_ELEM[L->field[g][k]];
        o = (o + e - 1) / e * e;
        offs[k] = o;
        o += member_bytes(L, g, k);
        if (e > al) al = e;
    }
    return (o + al - 1) / al * al;
}

/* Record size of group g and the offset of every member; returns -1 when g */
/* is out of range.  Used by tests to compare with ctypes structures.         */
int oracle_layout_group(int layout, uint64_t seed, int g, int32_t *nmem,
                        int32_t *fields, int32_t *comps, int32_t *offsets)
{
    layout_def L;
    if (build_layout(layout, seed, &L)) return -1;
    if (g < 0 || g >= L.ngroups) return -1;
    int offs[F_NUM];
    int rec = group_record(&L, g, offs);
    *nmem = L.nmem[g];
    for (int k = 0; k < L.nmem[g]; ++k) {
        fields[k] = L.field[g][k]; comps[k] = L.comp[g][k]; offsets[k] = offs[k];
    }
    return rec;
}

int oracle_layout_ngroups(int layout, uint64_t seed)
{
    layout_def L;
    if (build_layout(layout, seed, &L)) return -1;
    return L.ngroups;
}

int64_t oracle_store_bytes(int layout, uint64_t seed, int64_t n)
{
    layout_def L;
    if (build_layout(layout, seed, &L)) return -1;
    int64_t total = 0;
    for (int g = 0; g < L.ngroups; ++g) {
        int offs[F_NUM];
        total += round256(n * group_record(&L, g, offs));
    }
    return total;
}

static const uint8_t *field_src(const oracle_fields *f, int fid)
{
    switch (fid) {
    case F_X: return (const uint8_t *)f->x;
    case F_V: return (const uint8_t *)f->v;
    case F_A: return (const uint8_t *)f->a;
    case F_MASS: return (const uint8_t *)f->mass;
    case F_H: return (const uint8_t *)f->h;
    case F_U: return (const uint8_t *)f->u;
    case F_UDT: return (const uint8_t *)f->u_dt;
    case F_RHO: return (const uint8_t *)f->rho;
    case F_TBIN: return (const uint8_t *)f->time_bin;
    case F_AVISC: return (const uint8_t *)f->alpha_visc;
    case F_ADIFF: return (const uint8_t *)f->alpha_diff;
    case F_RHODH: return (const uint8_t *)f->rho_dh;
    case F_WCOUNT: return (const uint8_t *)f->wcount;
    case F_WCOUNTDH: return (const uint8_t *)f->wcount_dh;
    case F_DIVV: return (const uint8_t *)f->div_v;
    case F_ROTV: return (const uint8_t *)f->rot_v;
    case F_FGRADH: return (const uint8_t *)f->f_gradh;
    case F_PRES: return (const uint8_t *)f->pressure;
    case F_CS: return (const uint8_t *)f->soundspeed;
    case F_BALS: return (const uint8_t *)f->balsara;
    case F_VSIGG: return (const uint8_t *)f->v_sig_grad;
    case F_LAPU: return (const uint8_t *)f->laplace_u;
    case F_HDT: return (const uint8_t *)f->h_dt;
    case F_VSIG: return (const uint8_t *)f->v_sig;
    case F_ID: return (const uint8_t *)f->id;
    default: return NULL; /* ballast has no logical source: stays zero */
    }
}

/* Byte image of the store: particle k of the store is original particle   */
/* perm[k] (perm NULL: identity).  out must hold oracle_store_bytes bytes.  */
int oracle_store_encode(int layout, uint64_t seed, int64_t n,
                        const oracle_fields *f, const int64_t *perm, uint8_t *out)
{
    layout_def L;
    if (build_layout(layout, seed, &L)) return -1;
    int64_t base = 0;
    memset(out, 0, (size_t)oracle_store_bytes(layout, seed, n));
    for (int g = 0; g < L.ngroups; ++g) {
        int offs[F_NUM];
        int rec = group_record(&L, g, offs);
        for (int m = 0; m < L.nmem[g]; ++m) {
            int fid = L.field[g][m];
            const uint8_t *src = field_src(f, fid);
            if (!src) continue;
            int full = FIELD_ELEM[fid] * FIELD_COUNT[fid];
            int nb = member_bytes(&L, g, m);
            int coff = L.comp[g][m] >= 0 ? L.comp[g][m] * FIELD_ELEM[fid] : 0;
            for (int64_t k = 0; k < n; ++k) {
                int64_t p = perm ? perm[k] : k;
                memcpy(out + base + k * rec + offs[m], src + p * full + coff, (size_t)nb);
            }
        }
        base += round256(n * rec);
    }
    return 0;
}
