/*
 * loc_oracle.c -- plain FP64 CPU oracle of the LOC line radiative-transfer
 * hot path (Juvela, "LOC program for line radiative transfer").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two only see the
 * same seeded inputs.
 *
 * The method is an iteration (accelerated lambda iteration, ALI), so the
 * oracle performs the paper's steps in the paper's order, in the intensity
 * form that is algebraically equal to the paper's photon-count form:
 *   photons per ray and channel are I * A * Omega * dv / (h c)      (Eq. 1),
 *   the emission term of Eq. 3 with the s / sum(s) share (Sect. 2) equals
 *   S (1 - e^-tau) in intensity, and the external term of Eq. 2 is the
 *   path-averaged incoming intensity I_in (1 - e^-tau) / tau.
 * Intensities are occupation numbers n = I c^2 / (2 h nu^3).
 *
 * Each function says which passage it follows.  Where the paper is silent
 * the reading used is stated next to the code.
 *
 * Parity status: every function here is pinned by tests in tests/ against
 * closed forms, invariants or brute force (the per-cell line truncation by
 * tests/test_oracle_truncation.py), except one part, parity unpinned: the
 * exact intensity of octree side rays (bounded, not fixed: in a uniform
 * absorber they lie between the exact field and the field 2 h0 higher up;
 * the split rays at a refined cell's upstream face are pinned exactly) --
 * see the test module docstrings.  The infall line of a cloud with an
 * excitation gradient is pinned by its convergence to a fine numerical
 * integration of the continuous model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CGS constants (CODATA 2018 exact SI values). */
static const double LO_H = 6.62607015e-27;
static const double LO_KB = 1.380649e-16;
static const double LO_C = 2.99792458e10;
static const double LO_AMU = 1.66053906660e-24;
static const double LO_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Molecule                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n_levels, n_lines, n_coll;
    const double *energy_K, *g;
    double mass_amu;
    const int *line_u, *line_l;
    const double *line_A, *line_nu;
    const int *coll_u, *coll_l;
    const double *coll_k;
    /* hyperfine components of the lines (1D, Sect. 2.1), or hf_off = NULL:
     * line t's components are hf_off[t] .. hf_off[t+1]-1, each a velocity
     * offset hf_v (cm/s) and a relative strength hf_w (summing to 1); a line
     * with no components has the plain profile */
    const int *hf_off;
    const double *hf_v, *hf_w;
} lo_molecule;

/* Background occupation number of the cosmic background at temperature
 * t_bg for a line at nu: n = 1 / (exp(h nu / k T_bg) - 1) (Sect. 2, Eq. 1:
 * the rays enter carrying the background field). */
double lo_bg_occupation(double nu, double t_bg)
{
    if (t_bg <= 0.0) return 0.0;
    return 1.0 / expm1(LO_H * nu / (LO_KB * t_bg));
}

/* Boltzmann (LTE) populations at t_kin; the iteration starts from LTE
 * (Sect. 3.3.2).  x[i] = g_i exp(-E_i / T) / Z. */
void lo_lte_populations(int n_levels, const double *energy_K, const double *g,
                        int n_cells, const double *t_kin, double *x)
{
    for (int c = 0; c < n_cells; c++) {
        double z = 0.0;
        for (int i = 0; i < n_levels; i++) {
            x[c * n_levels + i] = g[i] * exp(-energy_K[i] / t_kin[c]);
            z += x[c * n_levels + i];
        }
        for (int i = 0; i < n_levels; i++) x[c * n_levels + i] /= z;
    }
}

/* ------------------------------------------------------------------------ */
/* Line profile: the share of the emitted photons falling in each channel   */
/* (Sect. 2, the practical form of the profile function).                   */
/* Gaussian of dispersion sigma integrated over channel k, whose velocity   */
/* interval is [v_min + k dv, v_min + (k+1) dv].  Gas moving with v_los     */
/* along the ray (towards the observer downstream) is blue-shifted, so the  */
/* local line centre sits at channel velocity -v_los.                       */
/* ------------------------------------------------------------------------ */
static double lo_upper_tail(double b)
{
    /* P(X > x) for a Gaussian with x = b * sqrt(2) sigma: 0.5 erfc(b). */
    return 0.5 * erfc(b);
}

void lo_profile(int n_ch, double v_min, double dv, double v_los, double sigma,
                double *phi)
{
    const double inv = 1.0 / (sqrt(2.0) * sigma);
    for (int k = 0; k < n_ch; k++) {
        double b0 = (v_min + k * dv + v_los) * inv;
        double b1 = (v_min + (k + 1) * dv + v_los) * inv;
        /* phi = Phi(b1) - Phi(b0) written with upper tails, which keeps
         * relative accuracy in both wings. */
        if (b0 >= 0.0)
            phi[k] = lo_upper_tail(b0) - lo_upper_tail(b1);
        else if (b1 <= 0.0)
            phi[k] = lo_upper_tail(-b1) - lo_upper_tail(-b0);
        else
            phi[k] = 1.0 - lo_upper_tail(-b0) - lo_upper_tail(b1);
    }
}

/* Profile of line t with hyperfine structure in LTE between its
 * components (Sect. 2.1; the relative populations of the components are
 * fixed, so the line is one transition whose profile is the
 * strength-weighted sum of the component profiles, each Doppler-shifted by
 * its velocity offset: a component at offset v_c appears at channel
 * velocity v_c - v_los).  phi0 is the unshifted profile; lines without
 * components take it as it is. */
static void lo_line_profile(const lo_molecule *m, int t, int n_ch, double v_min, double dv,
                            double v_los, double sigma, const double *phi0, double *phi_t, double *tmp)
{
    const int c0 = m->hf_off ? m->hf_off[t] : 0, c1 = m->hf_off ? m->hf_off[t + 1] : 0;
    if (c1 == c0) {
        memcpy(phi_t, phi0, sizeof(double) * n_ch);
        return;
    }
    for (int k = 0; k < n_ch; k++) phi_t[k] = 0.0;
    for (int c = c0; c < c1; c++) {
        lo_profile(n_ch, v_min, dv, v_los - m->hf_v[c], sigma, tmp);
        for (int k = 0; k < n_ch; k++) phi_t[k] += m->hf_w[c] * tmp[k];
    }
}

/* Total 1D line width: sigma^2 = sigma_turb^2 + k T / m (thermal plus
 * micro-turbulence; Sect. 3.3.1 counts thermal broadening in the width). */
static double lo_sigma(double sigma_turb, double t_kin, double mass_amu)
{
    return sqrt(sigma_turb * sigma_turb + LO_KB * t_kin / (mass_amu * LO_AMU));
}

/* ------------------------------------------------------------------------ */
/* Line parameters per cell and line (Eq. 2, Eq. 3).                         */
/*   tau_k = Kp * phi_k * s with                                             */
/*   Kp = c^3 A / (8 pi nu^3 dv) * n_mol * (x_l g_u / g_l - x_u)             */
/* (absorption coefficient (h nu / 4 pi)(n_l B_lu - n_u B_ul) phi_nu with    */
/* B_ul = A c^2 / (2 h nu^3), phi_nu = phi_k c / (nu dv)), and the source    */
/* function in occupation units S = 1 / (g_u x_l / (g_l x_u) - 1).           */
/* A vanishing population difference (|g_u x_l - g_l x_u| <= 1e-30 g_u x_l) */
/* gives Kp = 0, S = 0; inverted levels are kept as they are.                */
/* ------------------------------------------------------------------------ */
void lo_line_params(const lo_molecule *m, int n_cells, const double *n_h2,
                    const double *abundance, double dv, const double *x,
                    double *Kp, double *S)
{
    const int L = m->n_levels;
    for (int t = 0; t < m->n_lines; t++) {
        const int u = m->line_u[t], l = m->line_l[t];
        const double nu = m->line_nu[t];
        const double gu = m->g[u], gl = m->g[l];
        const double pre = LO_C * LO_C * LO_C * m->line_A[t] / (8.0 * LO_PI * nu * nu * nu * dv);
        for (int c = 0; c < n_cells; c++) {
            const double xl = x[c * L + l], xu = x[c * L + u];
            const double diff = gu * xl - gl * xu;
            const size_t o = (size_t)t * n_cells + c;
            if (fabs(diff) <= 1e-30 * gu * xl || (xl == 0.0 && xu == 0.0)) {
                Kp[o] = 0.0;
                S[o] = 0.0;
            } else {
                Kp[o] = pre * n_h2[c] * abundance[c] * diff / gl;
                S[o] = gl * xu / diff;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One step of a ray through one cell (Eq. 2, Eq. 3 in intensity form).      */
/* I[t][k] is the ray's intensity; the cell accumulators receive             */
/*   SIJ += w phi I f,   ESC += w phi f,   NORM += w phi                     */
/* with f = (1 - e^-tau) / tau (the external term of Eq. 2 and, through ESC, */
/* the local term that ALI drops, Sect. 2), and then                         */
/*   I <- I e^-tau + S (1 - e^-tau)                       (Eq. 3).           */
/* ------------------------------------------------------------------------ */
static void lo_step_lines(int n_lines, int n_ch, int n_cells, int cell,
                          const double *phi, const double *phi_lines, double s, double w,
                          const double *Kp, const double *S, double *I,
                          double *sij, double *esc, double *norm);

static void lo_step(int n_lines, int n_ch, int n_cells, int cell,
                    const double *phi, double s, double w,
                    const double *Kp, const double *S, double *I,
                    double *sij, double *esc, double *norm)
{
    lo_step_lines(n_lines, n_ch, n_cells, cell, phi, NULL, s, w, Kp, S, I, sij, esc, norm);
}

/* phi_lines: [n_lines][n_ch] per-line profiles (hyperfine), or NULL: every
 * line has phi.  NORM always sums the plain profile phi. */
static void lo_step_lines(int n_lines, int n_ch, int n_cells, int cell,
                          const double *phi, const double *phi_lines, double s, double w,
                          const double *Kp, const double *S, double *I,
                          double *sij, double *esc, double *norm)
{
    if (norm) {
        double sp = 0.0;
        for (int k = 0; k < n_ch; k++) sp += phi[k];
        norm[cell] += w * sp;
    }
    for (int t = 0; t < n_lines; t++) {
        const size_t o = (size_t)t * n_cells + cell;
        const double kp = Kp[o], src = S[o];
        const double *ph = phi_lines ? phi_lines + (size_t)t * n_ch : phi;
        double a_sij = 0.0, a_esc = 0.0;
        double *It = I + (size_t)t * n_ch;
        for (int k = 0; k < n_ch; k++) {
            const double tau = kp * ph[k] * s;
            const double one_m_e = -expm1(-tau);        /* 1 - e^-tau */
            const double f = (fabs(tau) < 1e-12) ? 1.0 - 0.5 * tau : one_m_e / tau;
            a_sij += ph[k] * It[k] * f;
            a_esc += ph[k] * f;
            It[k] = It[k] * (1.0 - one_m_e) + src * one_m_e;
        }
        if (sij) {
            sij[o] += w * a_sij;
            esc[o] += w * a_esc;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 1D geometry (Sect. 2.1): concentric shells with outer radii R_k; rays are */
/* parallel with impact parameters p; ray j of n_rays stands for the annulus */
/* between b_j = R (j / n_rays)^a and b_{j+1}, area A_j = pi (b_{j+1}^2 -   */
/* b_j^2), and passes at p_j = R ((j + 1/2) / n_rays)^a: equidistant rays    */
/* for a = 1 (the default), a power law otherwise (Sect. 2.1; our reading of */
/* the power-law option, which the paper does not spell out).  A ray with   */
/* impact parameter p                                                        */
/* visits shells K-1 .. t+1, the tangent shell t (smallest k with R_k > p)   */
/* in two halves, then t+1 .. K-1.  Path lengths are                         */
/*   s = sqrt(R_k^2 - p^2) - sqrt(R_{k-1}^2 - p^2),  tangent halves          */
/*   sqrt(R_t^2 - p^2).                                                      */
/* The Doppler shift is taken at the start of each step (Sect. 3.1):         */
/* v_los = v_k * cos(angle between radius vector and ray) at the entry       */
/* point; the outbound half of the tangent shell starts at cos = 0.          */
/* ------------------------------------------------------------------------ */
typedef struct { int cell; double s; double cosv; } lo_seg1d;

/* impact parameter and annulus area of ray j (a <= 0 means a = 1) */
static void lo_ray_1d(double Rout, int n_rays, double a, int j, double *p, double *A)
{
    if (!(a > 0.0)) a = 1.0;
    const double n = (double)n_rays;
    const double b0 = Rout * pow(j / n, a), b1 = Rout * pow((j + 1.0) / n, a);
    *p = Rout * pow((j + 0.5) / n, a);
    *A = LO_PI * (b1 * b1 - b0 * b0);
}

static int lo_tangent_shell(int K, const double *R, double p)
{
    for (int k = 0; k < K; k++) if (R[k] > p) return k;
    return K;
}

/* Fills segs (capacity >= 2K) for impact parameter p; returns count. */
static int lo_ray_segments_1d(int K, const double *R, double p, lo_seg1d *segs)
{
    const int t = lo_tangent_shell(K, R, p);
    int n = 0;
    if (t >= K) return 0;
    for (int k = K - 1; k > t; k--) {
        const double zo = sqrt(R[k] * R[k] - p * p);
        const double zi = sqrt(R[k - 1] * R[k - 1] - p * p);
        segs[n].cell = k; segs[n].s = zo - zi; segs[n].cosv = -zo / R[k]; n++;
    }
    const double zt = sqrt(R[t] * R[t] - p * p);
    segs[n].cell = t; segs[n].s = zt; segs[n].cosv = -zt / R[t]; n++;
    segs[n].cell = t; segs[n].s = zt; segs[n].cosv = 0.0; n++;
    for (int k = t + 1; k < K; k++) {
        const double zo = sqrt(R[k] * R[k] - p * p);
        const double zi = sqrt(R[k - 1] * R[k - 1] - p * p);
        segs[n].cell = k; segs[n].s = zo - zi; segs[n].cosv = zi / R[k - 1]; n++;
    }
    return n;
}

/* Exported for geometry tests: segment list of the equidistant ray j. */
int lo_paths_1d(int K, const double *R, int n_rays, double ray_power, int j,
                int *cell, double *s, double *cosv)
{
    const double Rout = R[K - 1];
    double p, A;
    lo_ray_1d(Rout, n_rays, ray_power, j, &p, &A);
    lo_seg1d *segs = (lo_seg1d *)malloc(sizeof(lo_seg1d) * 2 * (K + 1));
    int n = lo_ray_segments_1d(K, R, p, segs);
    for (int i = 0; i < n; i++) { cell[i] = segs[i].cell; s[i] = segs[i].s; cosv[i] = segs[i].cosv; }
    free(segs);
    return n;
}

/* Per-cell sum of A_j s over all rays: the "total length sum(s)" that turns
 * a ray's path length into its share of the cell's emission (Sect. 2). */
void lo_weights_1d(int K, const double *R, int n_rays, double ray_power, double *W)
{
    const double Rout = R[K - 1];
    lo_seg1d *segs = (lo_seg1d *)malloc(sizeof(lo_seg1d) * 2 * (K + 1));
    for (int c = 0; c < K; c++) W[c] = 0.0;
    for (int j = 0; j < n_rays; j++) {
        double p, A;
        lo_ray_1d(Rout, n_rays, ray_power, j, &p, &A);
        int n = lo_ray_segments_1d(K, R, p, segs);
        for (int i = 0; i < n; i++) W[segs[i].cell] += A * segs[i].s;
    }
    free(segs);
}

/* One radiation-field simulation over the 1D model (Sect. 2, 2.1): every
 * ray enters with the background, is followed through its shells with
 * lo_step, and each step's contribution carries the weight
 * w = A_j s / W_c (so that sum(w) = 1 per cell).  Outputs SIJ, ESC
 * [line][cell] and NORM [cell], zeroed here. */
/* The same ray simulation with a region of the k_sub innermost shells
 * (weights W_c from all n_rays rays in every mode):
 *   mode 0: all rays; each ray that reaches the region leaves in
 *           Ib[j][line][channel] the intensity it carries into it (before its
 *           first step inside the region);
 *   mode 1: only the rays j < j_end that reach the region, only their steps
 *           inside it, each starting from Ib[j]. */
void lo_march_1d_sub(const lo_molecule *m, int K, const double *R,
                     const double *t_kin, const double *sigma_turb,
                     const double *v, int n_ch, double v_min, double dv,
                     int n_rays, double ray_power, double t_bg, const double *Kp, const double *S,
                     int k_sub, int mode, int j_end, double *Ib,
                     double *SIJ, double *ESC, double *NORM);

void lo_march_1d(const lo_molecule *m, int K, const double *R,
                 const double *t_kin, const double *sigma_turb,
                 const double *v, int n_ch, double v_min, double dv,
                 int n_rays, double ray_power, double t_bg, const double *Kp, const double *S,
                 double *SIJ, double *ESC, double *NORM)
{
    lo_march_1d_sub(m, K, R, t_kin, sigma_turb, v, n_ch, v_min, dv, n_rays, ray_power, t_bg, Kp, S,
                    0, 0, n_rays, NULL, SIJ, ESC, NORM);
}

void lo_march_1d_sub(const lo_molecule *m, int K, const double *R,
                     const double *t_kin, const double *sigma_turb,
                     const double *v, int n_ch, double v_min, double dv,
                     int n_rays, double ray_power, double t_bg, const double *Kp, const double *S,
                     int k_sub, int mode, int j_end, double *Ib,
                     double *SIJ, double *ESC, double *NORM)
{
    if (mode == 0) j_end = n_rays;
    const int T = m->n_lines;
    const double Rout = R[K - 1];
    double *W = (double *)malloc(sizeof(double) * K);
    lo_weights_1d(K, R, n_rays, ray_power, W);
    memset(SIJ, 0, sizeof(double) * T * K);
    memset(ESC, 0, sizeof(double) * T * K);
    memset(NORM, 0, sizeof(double) * K);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthr * (2 * T + 1) * K, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *a_sij = acc + (size_t)tid * (2 * T + 1) * K;
        double *a_esc = a_sij + (size_t)T * K;
        double *a_norm = a_esc + (size_t)T * K;
        double *I = (double *)malloc(sizeof(double) * T * n_ch);
        double *phi = (double *)malloc(sizeof(double) * n_ch);
        double *phl = m->hf_off ? (double *)malloc(sizeof(double) * (T + 1) * n_ch) : NULL;
        lo_seg1d *segs = (lo_seg1d *)malloc(sizeof(lo_seg1d) * 2 * (K + 1));
#pragma omp for schedule(static)
        for (int j = 0; j < j_end; j++) {
            double p, A;
            lo_ray_1d(Rout, n_rays, ray_power, j, &p, &A);
            for (int t = 0; t < T; t++) {
                const double nbg = lo_bg_occupation(m->line_nu[t], t_bg);
                for (int k = 0; k < n_ch; k++) I[t * n_ch + k] = nbg;
            }
            int n = lo_ray_segments_1d(K, R, p, segs);
            /* the ray's steps inside the region: the middle 2 (K - k_sub) fewer */
            const int outer = (k_sub > 0) ? K - k_sub : 0;
            const int reaches = (k_sub > 0) && (n > 2 * outer);
            int i0 = 0, i1 = n;
            if (mode == 1) {
                i0 = outer;
                i1 = n - outer;
                memcpy(I, Ib + (size_t)j * T * n_ch, sizeof(double) * T * n_ch);
            }
            for (int i = i0; i < i1; i++) {
                if (mode == 0 && reaches && Ib && i == outer)
                    memcpy(Ib + (size_t)j * T * n_ch, I, sizeof(double) * T * n_ch);
                const int c = segs[i].cell;
                const double sig = lo_sigma(sigma_turb[c], t_kin[c], m->mass_amu);
                lo_profile(n_ch, v_min, dv, v[c] * segs[i].cosv, sig, phi);
                if (phl)
                    for (int t = 0; t < T; t++)
                        lo_line_profile(m, t, n_ch, v_min, dv, v[c] * segs[i].cosv, sig, phi,
                                        phl + (size_t)t * n_ch, phl + (size_t)T * n_ch);
                const double w = (W[c] > 0.0) ? A * segs[i].s / W[c] : 0.0;
                lo_step_lines(T, n_ch, K, c, phi, phl, segs[i].s, w, Kp, S, I, a_sij, a_esc, a_norm);
            }
        }
        free(I); free(phi); free(phl); free(segs);
    }
    for (int th = 0; th < nthr; th++) {
        const double *a = acc + (size_t)th * (2 * T + 1) * K;
        for (size_t i = 0; i < (size_t)T * K; i++) { SIJ[i] += a[i]; ESC[i] += a[(size_t)T * K + i]; }
        for (int c = 0; c < K; c++) NORM[c] += a[(size_t)2 * T * K + c];
    }
    free(acc);
    free(W);
}

/* ------------------------------------------------------------------------ */
/* Statistical equilibrium per cell (Sect. 2, ALI paragraph).                */
/* Radiative rates use the cell-averaged absorbed-photon counts in place of */
/* B_lu I_nu:  J_ext = SIJ / NORM, beta = ESC / NORM.  With ALI the local   */
/* term is left out and A_ul is scaled by beta:                              */
/*   R_lu = (g_u / g_l) A J_ext,   R_ul = A (beta + J_ext).                  */
/* Without ALI, J = J_ext + S (1 - beta) and beta = 1.                       */
/* Collisions: C_ul = n_H2 k_ul, C_lu = C_ul (g_u/g_l) exp(-(E_u-E_l)/T).    */
/* Row 0 of the balance equations is replaced by sum(x) = 1 and the system  */
/* is solved by Gaussian elimination with partial pivoting.                  */
/* If NORM = 0 (profile entirely outside the band) beta = 1, J_ext = n_bg.  */
/* ------------------------------------------------------------------------ */
static int lo_gauss_solve(int n, double *M, double *b)
{
    for (int p = 0; p < n; p++) {
        int piv = p;
        for (int i = p + 1; i < n; i++)
            if (fabs(M[i * n + p]) > fabs(M[piv * n + p])) piv = i;
        if (M[piv * n + p] == 0.0) return -1;
        if (piv != p) {
            for (int j = 0; j < n; j++) { double tmp = M[p * n + j]; M[p * n + j] = M[piv * n + j]; M[piv * n + j] = tmp; }
            double tb = b[p]; b[p] = b[piv]; b[piv] = tb;
        }
        for (int i = p + 1; i < n; i++) {
            const double f = M[i * n + p] / M[p * n + p];
            if (f == 0.0) continue;
            for (int j = p; j < n; j++) M[i * n + j] -= f * M[p * n + j];
            b[i] -= f * b[p];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double acc = b[i];
        for (int j = i + 1; j < n; j++) acc -= M[i * n + j] * b[j];
        b[i] = acc / M[i * n + i];
    }
    return 0;
}

/* Per-cell line truncation (Sect. 4 proposes computing, cell by cell, only   */
/* the transitions whose levels are populated, without giving a rule; this   */
/* is our reading): line t is off in cell c when both of its levels hold     */
/* less than `cutoff` of the molecules, off[t][c] = 1.  An off line has no   */
/* opacity in that cell (Kp = 0, S = 0: it neither absorbs nor emits there)  */
/* and its rates use the background field, J = n_bg with beta = 1.           */
void lo_line_off(const lo_molecule *m, int n_cells, const double *x, double cutoff,
                 unsigned char *off)
{
    const int L = m->n_levels;
    for (int t = 0; t < m->n_lines; t++) {
        const int u = m->line_u[t], l = m->line_l[t];
        for (int c = 0; c < n_cells; c++)
            off[(size_t)t * n_cells + c] =
                (cutoff > 0.0 && x[(size_t)c * L + l] < cutoff && x[(size_t)c * L + u] < cutoff) ? 1 : 0;
    }
}

/* off: [line][cell] truncation mask of lo_line_off, or NULL (none).
 * Solves cells [0, c_end) of the n_cells; the others are not written. */
static int lo_se_solve_range(const lo_molecule *m, int n_cells, int c_end, const double *n_h2,
                             const double *t_kin, double t_bg, int ali,
                             const double *SIJ, const double *ESC, const double *NORM,
                             const double *S, const unsigned char *off, double *x_out)
{
    const int L = m->n_levels, T = m->n_lines;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+:bad)
    for (int c = 0; c < c_end; c++) {
        double *R = (double *)calloc((size_t)L * L, sizeof(double)); /* R[i][j]: rate i -> j */
        double *M = (double *)calloc((size_t)L * L, sizeof(double));
        double *b = (double *)calloc(L, sizeof(double));
        for (int t = 0; t < T; t++) {
            const int u = m->line_u[t], l = m->line_l[t];
            const double A = m->line_A[t];
            const size_t o = (size_t)t * n_cells + c;
            double J, beta;
            if (off && off[o]) {
                J = lo_bg_occupation(m->line_nu[t], t_bg);
                beta = 1.0;
            } else if (NORM[c] > 0.0) {
                J = SIJ[o] / NORM[c];
                beta = ESC[o] / NORM[c];
            } else {
                J = lo_bg_occupation(m->line_nu[t], t_bg);
                beta = 1.0;
            }
            if (!ali) { J = J + S[o] * (1.0 - beta); beta = 1.0; }
            R[u * L + l] += A * (beta + J);
            R[l * L + u] += (m->g[u] / m->g[l]) * A * J;
        }
        for (int p = 0; p < m->n_coll; p++) {
            const int u = m->coll_u[p], l = m->coll_l[p];
            const double cul = n_h2[c] * m->coll_k[p];
            const double clu = cul * (m->g[u] / m->g[l]) * exp(-(m->energy_K[u] - m->energy_K[l]) / t_kin[c]);
            R[u * L + l] += cul;
            R[l * L + u] += clu;
        }
        /* balance of level i: sum_j x_j R[j][i] - x_i sum_j R[i][j] = 0 */
        for (int i = 0; i < L; i++) {
            double out = 0.0;
            for (int j = 0; j < L; j++) {
                if (j == i) continue;
                M[i * L + j] = R[j * L + i];
                out += R[i * L + j];
            }
            M[i * L + i] = -out;
        }
        for (int j = 0; j < L; j++) M[j] = 1.0;   /* row 0: sum(x) = 1 */
        b[0] = 1.0;
        if (lo_gauss_solve(L, M, b) != 0) bad++;
        for (int i = 0; i < L; i++) x_out[(size_t)c * L + i] = b[i];
        free(R); free(M); free(b);
    }
    return bad;
}

int lo_se_solve_off(const lo_molecule *m, int n_cells, const double *n_h2,
                    const double *t_kin, double t_bg, int ali,
                    const double *SIJ, const double *ESC, const double *NORM,
                    const double *S, const unsigned char *off, double *x_out)
{
    return lo_se_solve_range(m, n_cells, n_cells, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, off, x_out);
}

int lo_se_solve(const lo_molecule *m, int n_cells, const double *n_h2,
                const double *t_kin, double t_bg, int ali,
                const double *SIJ, const double *ESC, const double *NORM,
                const double *S, double *x_out)
{
    return lo_se_solve_off(m, n_cells, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, NULL, x_out);
}

/* Excitation temperature T_ex = (h nu / k) / ln(g_u x_l / (g_l x_u)),
 * [line][cell]; 0 where x_u = 0. */
void lo_tex(const lo_molecule *m, int n_cells, const double *x, double *tex)
{
    const int L = m->n_levels;
    for (int t = 0; t < m->n_lines; t++) {
        const int u = m->line_u[t], l = m->line_l[t];
        const double T0 = LO_H * m->line_nu[t] / LO_KB;
        for (int c = 0; c < n_cells; c++) {
            const double xu = x[(size_t)c * L + u], xl = x[(size_t)c * L + l];
            tex[(size_t)t * n_cells + c] = (xu > 0.0 && xl > 0.0)
                ? T0 / log(m->g[u] * xl / (m->g[l] * xu)) : 0.0;
        }
    }
}

/* Convergence metric: max over cells and lines with x_u >= 1e-6 of
 * |dT_ex| / |T_ex| between two population sets (Sect. 3.3.2 tracks T_ex). */
double lo_max_rel_dtex(const lo_molecule *m, int n_cells, const double *x_old,
                       const double *x_new)
{
    const int T = m->n_lines, L = m->n_levels;
    double *a = (double *)malloc(sizeof(double) * T * n_cells);
    double *b = (double *)malloc(sizeof(double) * T * n_cells);
    lo_tex(m, n_cells, x_old, a);
    lo_tex(m, n_cells, x_new, b);
    double mx = 0.0;
    for (int t = 0; t < T; t++)
        for (int c = 0; c < n_cells; c++) {
            const size_t o = (size_t)t * n_cells + c;
            if (x_new[(size_t)c * L + m->line_u[t]] < 1e-6) continue;
            if (a[o] == 0.0) continue;
            const double d = fabs(b[o] - a[o]) / fabs(a[o]);
            if (d > mx) mx = d;
        }
    free(a); free(b);
    return mx;
}

/* The ALI loop for a 1D model (Sect. 2): start from x (LTE or given),
 * then n_iter times: line parameters -> ray simulation -> equilibrium.
 * dtex[it] receives the per-iteration convergence metric.  cutoff > 0:
 * per-cell line truncation (lo_line_off) from each iteration's starting
 * populations. */
int lo_iterate_1d_cut(const lo_molecule *m, int K, const double *R,
                      const double *n_h2, const double *t_kin,
                      const double *sigma_turb, const double *abundance,
                      const double *v, int n_ch, double v_min, double dv,
                      int n_rays, double ray_power, double t_bg, int ali, int n_iter,
                      double cutoff, double *x, double *dtex)
{
    const int T = m->n_lines, L = m->n_levels;
    double *Kp = (double *)malloc(sizeof(double) * T * K);
    double *S = (double *)malloc(sizeof(double) * T * K);
    double *SIJ = (double *)malloc(sizeof(double) * T * K);
    double *ESC = (double *)malloc(sizeof(double) * T * K);
    double *NORM = (double *)malloc(sizeof(double) * K);
    double *xn = (double *)malloc(sizeof(double) * L * K);
    unsigned char *off = (unsigned char *)malloc((size_t)T * K);
    int bad = 0;
    for (int it = 0; it < n_iter; it++) {
        lo_line_params(m, K, n_h2, abundance, dv, x, Kp, S);
        lo_line_off(m, K, x, cutoff, off);
        for (size_t o = 0; o < (size_t)T * K; o++)
            if (off[o]) { Kp[o] = 0.0; S[o] = 0.0; }
        lo_march_1d(m, K, R, t_kin, sigma_turb, v, n_ch, v_min, dv, n_rays, ray_power, t_bg, Kp, S, SIJ, ESC, NORM);
        bad += lo_se_solve_off(m, K, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, off, xn);
        if (dtex) dtex[it] = lo_max_rel_dtex(m, K, x, xn);
        memcpy(x, xn, sizeof(double) * L * K);
    }
    free(Kp); free(S); free(SIJ); free(ESC); free(NORM); free(xn); free(off);
    return bad;
}

int lo_iterate_1d(const lo_molecule *m, int K, const double *R,
                  const double *n_h2, const double *t_kin,
                  const double *sigma_turb, const double *abundance,
                  const double *v, int n_ch, double v_min, double dv,
                  int n_rays, double ray_power, double t_bg, int ali, int n_iter,
                  double *x, double *dtex)
{
    return lo_iterate_1d_cut(m, K, R, n_h2, t_kin, sigma_turb, abundance, v, n_ch, v_min, dv,
                             n_rays, ray_power, t_bg, ali, n_iter, 0.0, x, dtex);
}

/* Rays that cross shells 0 .. k_sub - 1: the rays whose tangent shell is
 * below k_sub (impact parameters increase with j, so they are j < j_end). */
int lo_sub_rays_1d(int K, const double *R, int n_rays, double ray_power, int k_sub)
{
    const double Rout = R[K - 1];
    int j_end = 0;
    for (int j = 0; j < n_rays; j++) {
        double p, A;
        lo_ray_1d(Rout, n_rays, ray_power, j, &p, &A);
        if (lo_tangent_shell(K, R, p) < k_sub) j_end = j + 1;
    }
    return j_end;
}

/* ALI with sub-iterations on an inner region (Sect. 4 proposes updating the
 * populations of optically thick regions more often than the rest; the
 * scheme is our reading).  Each iteration is one full iteration (line
 * parameters, ray simulation of all rays, equilibrium of every cell)
 * followed by n_sub sub-iterations of the region of the k_sub innermost
 * shells: line parameters from the current populations, a ray simulation of
 * the rays that reach the region (every ray that crosses a region cell, so
 * the region's sums are complete) over their steps inside it, each ray
 * starting with the intensity it carried into the region in the full
 * iteration (the radiation entering the region is held), and the
 * equilibrium of the region's cells only; the populations outside the region
 * stay as the full iteration left them.  dtex[it] is the metric between the
 * populations before and after the whole iteration. */
int lo_iterate_1d_sub(const lo_molecule *m, int K, const double *R,
                      const double *n_h2, const double *t_kin,
                      const double *sigma_turb, const double *abundance,
                      const double *v, int n_ch, double v_min, double dv,
                      int n_rays, double ray_power, double t_bg, int ali, int n_iter,
                      int n_sub, int k_sub, double *x, double *dtex)
{
    const int T = m->n_lines, L = m->n_levels;
    double *Kp = (double *)malloc(sizeof(double) * T * K);
    double *S = (double *)malloc(sizeof(double) * T * K);
    double *SIJ = (double *)malloc(sizeof(double) * T * K);
    double *ESC = (double *)malloc(sizeof(double) * T * K);
    double *NORM = (double *)malloc(sizeof(double) * K);
    double *xn = (double *)malloc(sizeof(double) * L * K);
    double *x0 = (double *)malloc(sizeof(double) * L * K);
    const int j_end = lo_sub_rays_1d(K, R, n_rays, ray_power, k_sub);
    double *Ib = (double *)malloc(sizeof(double) * ((size_t)j_end + 1) * T * n_ch);
    int bad = 0;
    for (int it = 0; it < n_iter; it++) {
        memcpy(x0, x, sizeof(double) * L * K);
        lo_line_params(m, K, n_h2, abundance, dv, x, Kp, S);
        lo_march_1d_sub(m, K, R, t_kin, sigma_turb, v, n_ch, v_min, dv, n_rays, ray_power, t_bg, Kp, S,
                        k_sub, 0, n_rays, Ib, SIJ, ESC, NORM);
        bad += lo_se_solve_off(m, K, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, NULL, xn);
        memcpy(x, xn, sizeof(double) * L * K);
        for (int q = 0; q < n_sub; q++) {
            lo_line_params(m, K, n_h2, abundance, dv, x, Kp, S);
            lo_march_1d_sub(m, K, R, t_kin, sigma_turb, v, n_ch, v_min, dv, n_rays, ray_power, t_bg,
                            Kp, S, k_sub, 1, j_end, Ib, SIJ, ESC, NORM);
            bad += lo_se_solve_range(m, K, k_sub, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, NULL, xn);
            memcpy(x, xn, sizeof(double) * L * k_sub);     /* region cells only ([cell][level]) */
        }
        if (dtex) dtex[it] = lo_max_rel_dtex(m, K, x0, x);
    }
    free(Kp); free(S); free(SIJ); free(ESC); free(NORM); free(xn); free(x0); free(Ib);
    return bad;
}

/* Emergent spectra of a 1D model (Sect. 2: final line-of-sight integration
 * for a chosen line): for each impact parameter p the ray of the march
 * geometry is followed with fixed populations and no accumulation; output is
 * the Rayleigh-Jeans brightness T = (h nu / k)(n - n_bg) per channel. */
void lo_spectra_1d(const lo_molecule *m, int line, int K, const double *R,
                   const double *n_h2, const double *t_kin,
                   const double *sigma_turb, const double *abundance,
                   const double *v, int n_ch, double v_min, double dv,
                   double t_bg, const double *x, int n_p, const double *p,
                   double *T_out)
{
    const int T = m->n_lines;
    double *Kp = (double *)malloc(sizeof(double) * T * K);
    double *S = (double *)malloc(sizeof(double) * T * K);
    lo_line_params(m, K, n_h2, abundance, dv, x, Kp, S);
    const double nbg = lo_bg_occupation(m->line_nu[line], t_bg);
    const double T0 = LO_H * m->line_nu[line] / LO_KB;
#pragma omp parallel for schedule(dynamic)
    for (int ip = 0; ip < n_p; ip++) {
        double *I = (double *)malloc(sizeof(double) * n_ch);
        double *phi = (double *)malloc(sizeof(double) * n_ch);
        double *phl = (double *)malloc(sizeof(double) * 2 * n_ch);
        lo_seg1d *segs = (lo_seg1d *)malloc(sizeof(lo_seg1d) * 2 * (K + 1));
        for (int k = 0; k < n_ch; k++) I[k] = nbg;
        int n = lo_ray_segments_1d(K, R, p[ip], segs);
        for (int i = 0; i < n; i++) {
            const int c = segs[i].cell;
            const double sig = lo_sigma(sigma_turb[c], t_kin[c], m->mass_amu);
            lo_profile(n_ch, v_min, dv, v[c] * segs[i].cosv, sig, phi);
            lo_line_profile(m, line, n_ch, v_min, dv, v[c] * segs[i].cosv, sig, phi, phl, phl + n_ch);
            /* only line `line`: shift the parameter arrays to that row */
            lo_step(1, n_ch, K, c, phl, segs[i].s, 0.0, Kp + (size_t)line * K, S + (size_t)line * K, I, NULL, NULL, NULL);
        }
        for (int k = 0; k < n_ch; k++) T_out[(size_t)ip * n_ch + k] = T0 * (I[k] - nbg);
        free(I); free(phi); free(phl); free(segs);
    }
    free(Kp); free(S);
}

/* ------------------------------------------------------------------------ */
/* 3D geometry in integer fixed point (Sect. 2.2).                           */
/* The paper leaves the arithmetic open; this oracle defines the ray paths  */
/* exactly so that any implementation can reproduce them bit for bit:       */
/*  * one root cell is H0 = 2^F integer units; a level-L cell is H0 >> L.   */
/*  * the main axis m of direction d is argmax |d_i| (ties: lowest i); the  */
/*    transverse axes a < b are the other two.  Every axis with d_i < 0 is  */
/*    mirrored (x -> E - 1 - x, E = N H0) so the ray moves towards +m,+a,+b.*/
/*  * slopes q_a = floor(2^F |d_a| / |d_m| + 1/2) (likewise q_b).            */
/*  * lattice line (L, i, j) passes, at main-axis coordinate z in [0, E),   */
/*    through A(z) = o + i (H0 >> L) + floor(q_a z / 2^F)  (mod E) and      */
/*    B(z) = o + j (H0 >> L) + floor(q_b z / 2^F)  (mod E), with the common */
/*    offset o = (H0 >> Lmax) / 2 (periodic side faces, Sect. 2.2).         */
/*  * a segment is a maximal run of integers z with the same cell; its      */
/*    length is dz units, s = dz (h0 / 2^F) / |d_m|, and its weight is      */
/*    w = dz / ((H0 >> L_cell) n_dir), so every cell gets sum(w) = 1/n_dir  */
/*    per direction (constant path length per cell, Sect. 2.2).             */
/* On a regular grid all lines are level 0: one ray per upstream surface    */
/* element.                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int m, a, b;          /* main and transverse axes */
    int flip[3];          /* axis mirrored */
    int64_t qa, qb;       /* slopes in units of 2^-F */
} lo_dirinfo;

static void lo_direction_info(const double *d, int F, lo_dirinfo *di)
{
    int m = 0;
    if (fabs(d[1]) > fabs(d[m])) m = 1;
    if (fabs(d[2]) > fabs(d[m])) m = 2;
    di->m = m;
    di->a = (m == 0) ? 1 : 0;
    di->b = (m == 2) ? 1 : 2;
    for (int i = 0; i < 3; i++) di->flip[i] = d[i] < 0.0;
    const double scale = ldexp(1.0, F);
    di->qa = (int64_t)floor(scale * fabs(d[di->a]) / fabs(d[m]) + 0.5);
    di->qb = (int64_t)floor(scale * fabs(d[di->b]) / fabs(d[m]) + 0.5);
}

/* smallest z' > z at which floor(q z'/2^F) >= target (target > value at z) */
static int64_t lo_next_cross(int64_t q, int F, int64_t target)
{
    if (q <= 0) return INT64_MAX;
    const __int128 num = ((__int128)target) << F;
    return (int64_t)((num + q - 1) / q);
}

/* Exported for tests: direction decomposition. */
void lo_dir_info(const double *d, int F, int *m_ab_flip, int64_t *q)
{
    lo_dirinfo di;
    lo_direction_info(d, F, &di);
    m_ab_flip[0] = di.m; m_ab_flip[1] = di.a; m_ab_flip[2] = di.b;
    m_ab_flip[3] = di.flip[0]; m_ab_flip[4] = di.flip[1]; m_ab_flip[5] = di.flip[2];
    q[0] = di.qa; q[1] = di.qb;
}

/* Segments of root line (i, j) of a regular N^3 grid for one direction.
 * Writes cell index (x fastest), dz per segment; returns the count
 * (or -needed if cap is too small). */
static int64_t lo_line_segments_grid(int N, int F, const lo_dirinfo *di,
                                     int64_t i, int64_t j,
                                     int64_t *cells, int64_t *dzs, int64_t cap)
{
    const int64_t H = (int64_t)1 << F;
    const int64_t E = (int64_t)N * H;
    const int64_t o = H / 2;
    int64_t z = 0, n = 0;
    while (z < E) {
        const int64_t Au = o + i * H + (int64_t)(((__int128)di->qa * z) >> F);
        const int64_t Bu = o + j * H + (int64_t)(((__int128)di->qb * z) >> F);
        /* next boundary along each axis */
        int64_t zn = (z / H + 1) * H;
        const int64_t za = lo_next_cross(di->qa, F, (Au / H + 1) * H - o - i * H);
        const int64_t zb = lo_next_cross(di->qb, F, (Bu / H + 1) * H - o - j * H);
        if (za < zn) zn = za;
        if (zb < zn) zn = zb;
        if (zn > E) zn = E;
        /* mirrored integer coordinates -> original cell indices */
        int64_t pos[3];
        pos[di->m] = z;
        pos[di->a] = Au % E;
        pos[di->b] = Bu % E;
        int64_t ci[3];
        for (int ax = 0; ax < 3; ax++) {
            const int64_t pp = di->flip[ax] ? (E - 1 - pos[ax]) : pos[ax];
            ci[ax] = pp / H;
        }
        if (n < cap) {
            cells[n] = (ci[2] * N + ci[1]) * N + ci[0];
            dzs[n] = zn - z;
        }
        n++;
        z = zn;
    }
    return (n <= cap) ? n : -n;
}

int64_t lo_paths_grid3d(int N, int F, const double *d, int64_t i, int64_t j,
                        int64_t *cells, int64_t *dzs, int64_t cap)
{
    lo_dirinfo di;
    lo_direction_info(d, F, &di);
    return lo_line_segments_grid(N, F, &di, i, j, cells, dzs, cap);
}

/* One radiation-field simulation on a regular N^3 grid: n_dir directions,
 * N^2 root rays each, entering with the background (Sect. 2.2).  The per-
 * cell velocity is projected on the true direction; accumulators as in the
 * 1D case with w = dz / (H0 n_dir).  Directions [dir_lo, dir_hi) and root
 * rays with (i*N + j) % ray_stride == 0 are simulated (the stride only
 * serves bounded CPU timing samples; parity uses stride 1, all dirs). */
void lo_march_grid3d(const lo_molecule *m, int N, double h0, int F,
                     const double *t_kin, const double *sigma_turb,
                     const double *vx, const double *vy, const double *vz,
                     int n_dir, const double *dirs, int dir_lo, int dir_hi,
                     int ray_stride,
                     int n_ch, double v_min, double dv, double t_bg,
                     const double *Kp, const double *S,
                     double *SIJ, double *ESC, double *NORM)
{
    const int T = m->n_lines;
    const int64_t nc = (int64_t)N * N * N;
    const int64_t H = (int64_t)1 << F;
    memset(SIJ, 0, sizeof(double) * T * nc);
    memset(ESC, 0, sizeof(double) * T * nc);
    memset(NORM, 0, sizeof(double) * nc);
    /* One thread per line keeps the summation order fixed; thread of line 0
     * also accumulates NORM. */
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; t++) {
        const double nbg = lo_bg_occupation(m->line_nu[t], t_bg);
        double *I = (double *)malloc(sizeof(double) * n_ch);
        double *phi = (double *)malloc(sizeof(double) * n_ch);
        const int64_t cap = 4 * (int64_t)N + 16;
        int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * cap);
        int64_t *dzs = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *Kt = (double *)Kp + (size_t)t * nc;   /* this line's rows */
        double *St = (double *)S + (size_t)t * nc;
        for (int id = dir_lo; id < dir_hi; id++) {
            const double *d = dirs + 3 * id;
            lo_dirinfo di;
            lo_direction_info(d, F, &di);
            const double unit = h0 / (double)H / fabs(d[di.m]);
            for (int64_t i = 0; i < N; i++)
                for (int64_t j = 0; j < N; j++) {
                    if ((i * N + j) % ray_stride) continue;
                    for (int k = 0; k < n_ch; k++) I[k] = nbg;
                    const int64_t n = lo_line_segments_grid(N, F, &di, i, j, cells, dzs, cap);
                    for (int64_t sidx = 0; sidx < n; sidx++) {
                        const int64_t c = cells[sidx];
                        const double sig = lo_sigma(sigma_turb[c], t_kin[c], m->mass_amu);
                        const double vlos = vx[c] * d[0] + vy[c] * d[1] + vz[c] * d[2];
                        lo_profile(n_ch, v_min, dv, vlos, sig, phi);
                        const double s = (double)dzs[sidx] * unit;
                        const double w = (double)dzs[sidx] / ((double)H * n_dir);
                        /* single-line step on this line's rows */
                        double sij1 = 0.0, esc1 = 0.0;
                        lo_step(1, n_ch, 1, 0, phi, s, w, Kt + c, St + c, I, &sij1, &esc1, (t == 0) ? NORM + c : NULL);
                        SIJ[(size_t)t * nc + c] += sij1;
                        ESC[(size_t)t * nc + c] += esc1;
                    }
                }
        }
        free(I); free(phi); free(cells); free(dzs);
    }
}

/* ALI loop on a regular grid (as lo_iterate_1d). */
int lo_iterate_grid3d(const lo_molecule *m, int N, double h0, int F,
                      const double *n_h2, const double *t_kin,
                      const double *sigma_turb, const double *abundance,
                      const double *vx, const double *vy, const double *vz,
                      int n_dir, const double *dirs, int n_ch, double v_min,
                      double dv, double t_bg, int ali, int n_iter,
                      double *x, double *dtex)
{
    const int T = m->n_lines, L = m->n_levels;
    const int64_t nc = (int64_t)N * N * N;
    double *Kp = (double *)malloc(sizeof(double) * T * nc);
    double *S = (double *)malloc(sizeof(double) * T * nc);
    double *SIJ = (double *)malloc(sizeof(double) * T * nc);
    double *ESC = (double *)malloc(sizeof(double) * T * nc);
    double *NORM = (double *)malloc(sizeof(double) * nc);
    double *xn = (double *)malloc(sizeof(double) * L * nc);
    int bad = 0;
    for (int it = 0; it < n_iter; it++) {
        lo_line_params(m, (int)nc, n_h2, abundance, dv, x, Kp, S);
        lo_march_grid3d(m, N, h0, F, t_kin, sigma_turb, vx, vy, vz, n_dir, dirs, 0, n_dir, 1,
                        n_ch, v_min, dv, t_bg, Kp, S, SIJ, ESC, NORM);
        bad += lo_se_solve(m, (int)nc, n_h2, t_kin, t_bg, ali, SIJ, ESC, NORM, S, xn);
        if (dtex) dtex[it] = lo_max_rel_dtex(m, (int)nc, x, xn);
        memcpy(x, xn, sizeof(double) * L * nc);
    }
    free(Kp); free(S); free(SIJ); free(ESC); free(NORM); free(xn);
    return bad;
}


/* ------------------------------------------------------------------------ */
/* 3D octree grids (Sect. 2.2).                                              */
/* Cells are level ordered: level-0 cells in raster order (x fastest), then */
/* the 8 children (octant cx + 2 cy + 4 cz) of every refined level-L cell,   */
/* in the order of their parents.  A level-L cell is H0 >> L units wide.     */
/*                                                                           */
/* Reading of the ray rules (split rays at the upstream border of a refined  */
/* cell, side rays, recursive splitting, termination on coarsening, periodic */
/* re-entry): lattice lines exist at every level L, at                       */
/* A(z) = o + i (H0 >> L) + floor(q_a z / 2^F) with the common offset        */
/* o = (H0 >> Lmax) / 2, so the level-L lattice contains the level-(L-1) one.*/
/* A line's creation level lambda is the coarsest level whose lattice holds  */
/* it.  A line is active in a leaf iff the leaf's level >= lambda: then every*/
/* level-L leaf is crossed by exactly the level-L lattice, which is what the */
/* split, side and termination rules achieve, and the path length per cell  */
/* and direction is exactly H_L.  A line that becomes active on entering a  */
/* leaf c (after being inactive, or at the model's upstream face) starts     */
/* with the intensity of its parent: the level-(lambda-1) lattice line that  */
/* crosses the upstream face of C, the level-(lambda-1) ancestor of c, taken */
/* where it crosses that face (for lambda = 0: the background).  Photon     */
/* splitting into 1/4 and scaling by 4^-dL on termination leave the          */
/* intensity unchanged.                                                      */
/*                                                                           */
/* The oracle walks every lattice line of every level through the whole    */
/* model (pass 1: segments, activation events and parents), then follows    */
/* the lines in order of creation level (pass 2), so a parent's intensity at */
/* each requested face is known before its children start.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N, Lmax, F;
    int64_t n_cells;
    int64_t *child;       /* first child or -1 */
} lo_tree;

static int lo_tree_build(lo_tree *t, int N, int Lmax, int F, int64_t n_cells, const int32_t *refine)
{
    t->N = N; t->Lmax = Lmax; t->F = F; t->n_cells = n_cells;
    t->child = (int64_t *)malloc(sizeof(int64_t) * n_cells);
    int64_t nxt = (int64_t)N * N * N;
    for (int64_t c = 0; c < n_cells; c++) {
        if (refine[c]) { t->child[c] = nxt; nxt += 8; }
        else t->child[c] = -1;
    }
    return (nxt == n_cells) ? 0 : -1;
}

/* leaf containing the original-coordinate point; *level receives its level */
static int64_t lo_tree_locate(const lo_tree *t, int64_t x, int64_t y, int64_t z, int max_level, int *level)
{
    const int F = t->F, N = t->N;
    int64_t c = ((z >> F) * N + (y >> F)) * N + (x >> F);
    int L = 0;
    while (t->child[c] >= 0 && L < max_level) {
        L++;
        const int sh = F - L;
        const int oct = (int)(((x >> sh) & 1) | (((y >> sh) & 1) << 1) | (((z >> sh) & 1) << 2));
        c = t->child[c] + oct;
    }
    *level = L;
    return c;
}

typedef struct { int64_t z0, dz, cell; int level, active; } lo_oseg;
typedef struct { int lam; int64_t i, j, seg0, nseg; } lo_oline;
typedef struct { int64_t line, seg, parent, z_face, snap; } lo_oevent;

typedef struct {
    lo_oline *lines; int64_t n_lines;
    lo_oseg *segs; int64_t n_segs, cap_segs;
    lo_oevent *ev; int64_t n_ev, cap_ev;
    int64_t **table;      /* [lambda][i * M + j] -> line id (-1 for coarser lines) */
} lo_odir;

/* mirrored coordinates (ray moving +m, +a, +b) -> original, per axis */
static int64_t lo_unmirror(const lo_dirinfo *di, int ax, int64_t v, int64_t E)
{
    return di->flip[ax] ? E - 1 - v : v;
}

/* original-axis cell lower corner -> mirrored lower corner */
static int64_t lo_mirror_lo(const lo_dirinfo *di, int ax, int64_t lo, int64_t H, int64_t E)
{
    return di->flip[ax] ? E - lo - H : lo;
}

static void lo_point(const lo_dirinfo *di, int64_t z, int64_t Au, int64_t Bu, int64_t E, int64_t p[3])
{
    int64_t m[3];
    m[di->m] = z; m[di->a] = Au % E; m[di->b] = Bu % E;
    for (int ax = 0; ax < 3; ax++) p[ax] = lo_unmirror(di, ax, m[ax], E);
}

static int64_t lo_floorq(int64_t q, int64_t z, int F) { return (int64_t)(((__int128)q * z) >> F); }

static void lo_push_seg(lo_odir *D, lo_oseg sg)
{
    if (D->n_segs == D->cap_segs) {
        D->cap_segs = D->cap_segs ? 2 * D->cap_segs : 4096;
        D->segs = (lo_oseg *)realloc(D->segs, sizeof(lo_oseg) * D->cap_segs);
    }
    D->segs[D->n_segs++] = sg;
}

static void lo_push_ev(lo_odir *D, lo_oevent e)
{
    if (D->n_ev == D->cap_ev) {
        D->cap_ev = D->cap_ev ? 2 * D->cap_ev : 1024;
        D->ev = (lo_oevent *)realloc(D->ev, sizeof(lo_oevent) * D->cap_ev);
    }
    D->ev[D->n_ev++] = e;
}

/* walk line (lam, i, j) from z = 0 to E through the leaves, appending segments */
static void lo_walk_octree_line(const lo_tree *t, const lo_dirinfo *di, int lam, int64_t i, int64_t j, lo_odir *D)
{
    const int F = t->F;
    const int64_t H0 = (int64_t)1 << F;
    const int64_t E = (int64_t)t->N * H0;
    const int64_t o = (H0 >> t->Lmax) / 2;
    const int64_t A0 = o + i * (H0 >> lam), B0 = o + j * (H0 >> lam);
    int64_t z = 0;
    while (z < E) {
        const int64_t Au = A0 + lo_floorq(di->qa, z, F);
        const int64_t Bu = B0 + lo_floorq(di->qb, z, F);
        int64_t p[3];
        lo_point(di, z, Au, Bu, E, p);
        int L;
        const int64_t c = lo_tree_locate(t, p[0], p[1], p[2], t->Lmax, &L);
        const int64_t HL = H0 >> L;
        int64_t mlo[3];
        for (int ax = 0; ax < 3; ax++) mlo[ax] = lo_mirror_lo(di, ax, (p[ax] / HL) * HL, HL, E);
        int64_t zn = mlo[di->m] + HL;
        {
            const int64_t am = Au % E;
            const int64_t target = Au - am + mlo[di->a] + HL - A0;
            const int64_t za = lo_next_cross(di->qa, F, target);
            if (za < zn) zn = za;
        }
        {
            const int64_t bm = Bu % E;
            const int64_t target = Bu - bm + mlo[di->b] + HL - B0;
            const int64_t zb = lo_next_cross(di->qb, F, target);
            if (zb < zn) zn = zb;
        }
        if (zn > E) zn = E;
        lo_oseg sg = {z, zn - z, c, L, L >= lam};
        lo_push_seg(D, sg);
        z = zn;
    }
}

static int lo_creation_level(int lam, int64_t i, int64_t j)
{
    while (lam > 0 && (i % 2) == 0 && (j % 2) == 0) { lam--; i /= 2; j /= 2; }
    return lam;
}

/* pass 1 for one direction */
static void lo_octree_geometry(const lo_tree *t, const double *d, lo_odir *D)
{
    memset(D, 0, sizeof(*D));
    lo_dirinfo di;
    lo_direction_info(d, t->F, &di);
    const int F = t->F, Lmax = t->Lmax;
    const int64_t H0 = (int64_t)1 << F;
    const int64_t E = (int64_t)t->N * H0;
    const int64_t o = (H0 >> Lmax) / 2;
    /* line ids in order of creation level */
    D->table = (int64_t **)malloc(sizeof(int64_t *) * (Lmax + 1));
    int64_t nl = 0;
    for (int lam = 0; lam <= Lmax; lam++) {
        const int64_t M = (int64_t)t->N << lam;
        D->table[lam] = (int64_t *)malloc(sizeof(int64_t) * M * M);
        for (int64_t i = 0; i < M; i++)
            for (int64_t j = 0; j < M; j++)
                D->table[lam][i * M + j] = (lo_creation_level(lam, i, j) == lam) ? nl++ : -1;
    }
    D->n_lines = nl;
    D->lines = (lo_oline *)malloc(sizeof(lo_oline) * nl);
    for (int lam = 0; lam <= Lmax; lam++) {
        const int64_t M = (int64_t)t->N << lam;
        for (int64_t i = 0; i < M; i++)
            for (int64_t j = 0; j < M; j++) {
                const int64_t id = D->table[lam][i * M + j];
                if (id < 0) continue;
                lo_oline *ln = &D->lines[id];
                ln->lam = lam; ln->i = i; ln->j = j;
                ln->seg0 = D->n_segs;
                lo_walk_octree_line(t, &di, lam, i, j, D);
                ln->nseg = D->n_segs - ln->seg0;
            }
    }
    /* activation events */
    for (int64_t id = 0; id < nl; id++) {
        const lo_oline *ln = &D->lines[id];
        for (int64_t k = 0; k < ln->nseg; k++) {
            const lo_oseg *sg = &D->segs[ln->seg0 + k];
            if (!sg->active) continue;
            if (k > 0 && D->segs[ln->seg0 + k - 1].active) continue;
            lo_oevent e = {id, ln->seg0 + k, -1, 0, D->n_ev};
            if (ln->lam > 0) {
                const int lp = ln->lam - 1;
                const int64_t Hp = H0 >> lp;
                const int64_t Au = o + ln->i * (H0 >> ln->lam) + lo_floorq(di.qa, sg->z0, F);
                const int64_t Bu = o + ln->j * (H0 >> ln->lam) + lo_floorq(di.qb, sg->z0, F);
                int64_t p[3];
                lo_point(&di, sg->z0, Au, Bu, E, p);
                int Lc;
                const int64_t C = lo_tree_locate(t, p[0], p[1], p[2], lp, &Lc);
                (void)C;
                int64_t mlo[3];
                for (int ax = 0; ax < 3; ax++) mlo[ax] = lo_mirror_lo(&di, ax, (p[ax] / Hp) * Hp, Hp, E);
                const int64_t zf = mlo[di.m];
                const int64_t Mp = (int64_t)t->N << lp;
                int64_t Da = (mlo[di.a] - o - lo_floorq(di.qa, zf, F)) % E; if (Da < 0) Da += E;
                int64_t Db = (mlo[di.b] - o - lo_floorq(di.qb, zf, F)) % E; if (Db < 0) Db += E;
                int64_t ip = ((Da + Hp - 1) / Hp) % Mp, jp = ((Db + Hp - 1) / Hp) % Mp;
                int lpp = lp;
                while (lpp > 0 && (ip % 2) == 0 && (jp % 2) == 0) { lpp--; ip /= 2; jp /= 2; }
                e.parent = D->table[lpp][ip * ((int64_t)t->N << lpp) + jp];
                e.z_face = zf;
            }
            lo_push_ev(D, e);
        }
    }
}

static void lo_odir_free(lo_odir *D, int Lmax)
{
    for (int lam = 0; lam <= Lmax; lam++) free(D->table[lam]);
    free(D->table); free(D->lines); free(D->segs); free(D->ev);
}

/* Exported for tests: number of lines and segments of a direction, and the
 * segments (z0, dz, cell, level, active) of line (lam, i, j). */
int64_t lo_octree_line_segments(int N, int Lmax, int F, int64_t n_cells, const int32_t *refine,
                                const double *d, int lam, int64_t i, int64_t j, int64_t *out5, int64_t cap)
{
    lo_tree t;
    if (lo_tree_build(&t, N, Lmax, F, n_cells, refine) != 0) { free(t.child); return -1; }
    lo_dirinfo di;
    lo_direction_info(d, F, &di);
    lo_odir D;
    memset(&D, 0, sizeof(D));
    lo_walk_octree_line(&t, &di, lam, i, j, &D);
    const int64_t n = D.n_segs;
    for (int64_t k = 0; k < n && k < cap; k++) {
        out5[5 * k + 0] = D.segs[k].z0; out5[5 * k + 1] = D.segs[k].dz; out5[5 * k + 2] = D.segs[k].cell;
        out5[5 * k + 3] = D.segs[k].level; out5[5 * k + 4] = D.segs[k].active;
    }
    free(D.segs); free(t.child);
    return n;
}

/* Exported for tests: per-cell sum of active main-axis path over all lines of
 * one direction (int64 [n_cells]); returns the number of active segments. */
int64_t lo_octree_path_sums(int N, int Lmax, int F, int64_t n_cells, const int32_t *refine,
                            const double *d, int64_t *sum_dz)
{
    lo_tree t;
    if (lo_tree_build(&t, N, Lmax, F, n_cells, refine) != 0) { free(t.child); return -1; }
    lo_odir D;
    lo_octree_geometry(&t, d, &D);
    memset(sum_dz, 0, sizeof(int64_t) * n_cells);
    int64_t na = 0;
    for (int64_t k = 0; k < D.n_segs; k++)
        if (D.segs[k].active) { sum_dz[D.segs[k].cell] += D.segs[k].dz; na++; }
    lo_odir_free(&D, Lmax);
    free(t.child);
    return na;
}

/* One radiation-field simulation on an octree (Sect. 2.2).  Per-cell arrays
 * are level ordered over all cells (values of refined cells unused);
 * outputs SIJ, ESC [line][cell] and NORM [cell] (zero on refined cells).
 * Returns 0, or -1 for an inconsistent refinement array. */
int lo_march_octree(const lo_molecule *m, int N, int Lmax, int F, int64_t n_cells, const int32_t *refine,
                    double h0, const double *t_kin, const double *sigma_turb,
                    const double *vx, const double *vy, const double *vz,
                    int n_dir, const double *dirs, int n_ch, double v_min, double dv, double t_bg,
                    const double *Kp, const double *S, double *SIJ, double *ESC, double *NORM)
{
    const int T = m->n_lines;
    lo_tree t;
    if (lo_tree_build(&t, N, Lmax, F, n_cells, refine) != 0) { free(t.child); return -1; }
    const int64_t H0 = (int64_t)1 << F;
    memset(SIJ, 0, sizeof(double) * T * n_cells);
    memset(ESC, 0, sizeof(double) * T * n_cells);
    memset(NORM, 0, sizeof(double) * n_cells);
    for (int id = 0; id < n_dir; id++) {
        const double *d = dirs + 3 * id;
        lo_dirinfo di;
        lo_direction_info(d, F, &di);
        const double unit = h0 / (double)H0 / fabs(d[di.m]);
        lo_odir D;
        lo_octree_geometry(&t, d, &D);
        /* snapshot requests per parent line, and each event's snapshot slot */
        int64_t *req_n = (int64_t *)calloc(D.n_lines + 1, sizeof(int64_t));
        for (int64_t e = 0; e < D.n_ev; e++) if (D.ev[e].parent >= 0) req_n[D.ev[e].parent + 1]++;
        for (int64_t l = 0; l < D.n_lines; l++) req_n[l + 1] += req_n[l];
        int64_t *req_ev = (int64_t *)malloc(sizeof(int64_t) * (D.n_ev + 1));
        int64_t *fill = (int64_t *)calloc(D.n_lines, sizeof(int64_t));
        for (int64_t e = 0; e < D.n_ev; e++) {
            const int64_t p = D.ev[e].parent;
            if (p >= 0) req_ev[req_n[p] + fill[p]++] = e;
        }
        /* event index of each segment that starts an active interval */
        int64_t *seg_ev = (int64_t *)malloc(sizeof(int64_t) * (D.n_segs + 1));
        for (int64_t k = 0; k < D.n_segs; k++) seg_ev[k] = -1;
        for (int64_t e = 0; e < D.n_ev; e++) seg_ev[D.ev[e].seg] = e;
#pragma omp parallel for schedule(dynamic, 1)
        for (int tt = 0; tt < T; tt++) {
            const double nbg = lo_bg_occupation(m->line_nu[tt], t_bg);
            double *snap = (double *)malloc(sizeof(double) * (D.n_ev + 1) * n_ch);
            double *I = (double *)malloc(sizeof(double) * n_ch);
            double *phi = (double *)malloc(sizeof(double) * n_ch);
            for (int64_t l = 0; l < D.n_lines; l++) {      /* lines are in creation-level order */
                const lo_oline *ln = &D.lines[l];
                for (int k = 0; k < n_ch; k++) I[k] = nbg;
                for (int64_t q = 0; q < ln->nseg; q++) {
                    const int64_t sk = ln->seg0 + q;
                    const lo_oseg *sg = &D.segs[sk];
                    const int64_t e = seg_ev[sk];
                    if (e >= 0) {                           /* activation */
                        if (D.ev[e].parent < 0) for (int k = 0; k < n_ch; k++) I[k] = nbg;
                        else for (int k = 0; k < n_ch; k++) I[k] = snap[D.ev[e].snap * n_ch + k];
                    }
                    if (!sg->active) continue;
                    /* children waiting for this line's intensity at this face */
                    for (int64_t r = req_n[l]; r < req_n[l + 1]; r++) {
                        const int64_t ce = req_ev[r];
                        if (D.ev[ce].z_face == sg->z0)
                            for (int k = 0; k < n_ch; k++) snap[ce * n_ch + k] = I[k];
                    }
                    const int64_t c = sg->cell;
                    const double sig = lo_sigma(sigma_turb[c], t_kin[c], m->mass_amu);
                    const double vlos = vx[c] * d[0] + vy[c] * d[1] + vz[c] * d[2];
                    lo_profile(n_ch, v_min, dv, vlos, sig, phi);
                    const double s = (double)sg->dz * unit;
                    const double w = (double)sg->dz / ((double)(H0 >> sg->level) * n_dir);
                    double sij1 = 0.0, esc1 = 0.0;
                    lo_step(1, n_ch, 1, 0, phi, s, w, Kp + (size_t)tt * n_cells + c, S + (size_t)tt * n_cells + c,
                            I, &sij1, &esc1, NULL);
                    SIJ[(size_t)tt * n_cells + c] += sij1;
                    ESC[(size_t)tt * n_cells + c] += esc1;
                    if (tt == 0) {
                        double sp = 0.0;
                        for (int k = 0; k < n_ch; k++) sp += phi[k];
                        NORM[c] += w * sp;
                    }
                }
            }
            free(snap); free(I); free(phi);
        }
        /* every event must have received its snapshot (parent active at the face) */
        free(req_n); free(req_ev); free(fill); free(seg_ev);
        lo_odir_free(&D, Lmax);
    }
    free(t.child);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Emergent map of a 3D model (Sect. 2: after convergence the line of sight */
/* is integrated for chosen transitions; Sect. 3.3 shows such maps).  The   */
/* map is seen along direction d: one pixel per lattice line (lam, i, j) of */
/* that direction (i along the first transverse axis a, j along b; M =      */
/* N << lam pixels per side; lam = 0 for a regular grid).  The pixel's ray  */
/* starts with the background at the upstream face and crosses the periodic */
/* model once along the main axis, through every cell it meets -- every     */
/* leaf of an octree, whatever its level (an observer's line of sight; the  */
/* activation rules of the ray simulation do not apply) -- with the         */
/* intensity update of Eq. 3 and no accumulation.  Output, pixels with      */
/* (i M + j) % pix_stride == 0 (others untouched):                          */
/*   T[(i M + j) n_ch + k] = (h nu / k) (I_k - n_bg)   for line `line`.     */
/* A regular grid is the tree with Lmax = 0 and no refined cell.  Per-cell  */
/* arrays and Kp, S [line][cell] are level ordered over all cells.  Returns */
/* 0, or -1 for an inconsistent refinement array.                          */
/* ------------------------------------------------------------------------ */
int lo_map_3d(const lo_molecule *m, int line, int N, int Lmax, int F, int64_t n_cells,
              const int32_t *refine, double h0, const double *t_kin, const double *sigma_turb,
              const double *vx, const double *vy, const double *vz, const double *d, int lam,
              int64_t pix_stride, int n_ch, double v_min, double dv, double t_bg,
              const double *Kp, const double *S, double *T)
{
    lo_tree t;
    if (lo_tree_build(&t, N, Lmax, F, n_cells, refine) != 0) { free(t.child); return -1; }
    lo_dirinfo di;
    lo_direction_info(d, F, &di);
    const double unit = h0 / ldexp(1.0, F) / fabs(d[di.m]);
    const double nbg = lo_bg_occupation(m->line_nu[line], t_bg);
    const double T0 = LO_H * m->line_nu[line] / LO_KB;
    const int64_t M = (int64_t)N << lam;
    const double *Kt = Kp + (size_t)line * n_cells;
    const double *St = S + (size_t)line * n_cells;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t pix = 0; pix < M * M; pix++) {
        if (pix % pix_stride) continue;
        lo_odir D;
        memset(&D, 0, sizeof(D));
        lo_walk_octree_line(&t, &di, lam, pix / M, pix % M, &D);
        double *I = (double *)malloc(sizeof(double) * n_ch);
        double *phi = (double *)malloc(sizeof(double) * n_ch);
        for (int k = 0; k < n_ch; k++) I[k] = nbg;
        for (int64_t q = 0; q < D.n_segs; q++) {
            const int64_t c = D.segs[q].cell;
            const double sig = lo_sigma(sigma_turb[c], t_kin[c], m->mass_amu);
            const double vlos = vx[c] * d[0] + vy[c] * d[1] + vz[c] * d[2];
            lo_profile(n_ch, v_min, dv, vlos, sig, phi);
            lo_step(1, n_ch, 1, 0, phi, (double)D.segs[q].dz * unit, 0.0, Kt + c, St + c, I,
                    NULL, NULL, NULL);
        }
        for (int k = 0; k < n_ch; k++) T[pix * n_ch + k] = T0 * (I[k] - nbg);
        free(I); free(phi); free(D.segs);
    }
    free(t.child);
    return 0;
}

int lo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
