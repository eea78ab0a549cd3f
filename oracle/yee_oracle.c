/*
 * Plain FP64 Yee FDTD for one source simulation of the time-domain Casimir
 * method (McCauley, Rodriguez, Joannopoulos, Johnson, "Casimir forces in the
 * time domain: Applications", arXiv:0906.5170).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the CPU oracle against which the
 * CUDA path is checked.  Only tests, the smoke check and the benchmark's CPU
 * baseline load it; the product never does.  It shares no code with the CUDA
 * path.
 *
 * What one call computes (Sec. II; Eq. (1) and the definition of Gamma^E_i):
 *   - a harmonic source J = delta(t) f_n (or its magnetic dual K) on the
 *     stress surface S, given here as the post-impulse flux D(0+) (or B(0+));
 *   - the Yee leapfrog (Sec. III A: the FDTD code of the paper works on a Yee
 *     grid) in a medium whose contour conductivity sigma (Sec. II) sits on D
 *     for J sources and on B for K sources;
 *   - optional CPML absorbing layers (Sec. III B), Bloch-periodic wrap
 *     (Sec. III B, III D), z-invariance with d/dz -> i k_z (Sec. III B),
 *     and single-pole Lorentz media by an auxiliary differential equation
 *     analytically continued onto the contour (Sec. III B, Eq. (9));
 *   - at every step n = 1..T the surface functional s(n) = sum_m w_m F[c_m][i_m]
 *     of the measured field F (E for J sources, H for K sources).
 *
 * Fields are complex double (or real double in the ORACLE_REAL build), updated
 * by plain loops over every cell.
 *
 * Layout: every array is [k][j][i] with i fastest, index (k*ny + j)*nx + i.
 * Component sites (in units of Delta): E_x (i+1/2, j, k), E_y (i, j+1/2, k),
 * E_z (i, j, k+1/2); H_x (i, j+1/2, k+1/2), H_y (i+1/2, j, k+1/2),
 * H_z (i+1/2, j+1/2, k).  Indices wrap around each axis; a Bloch axis
 * multiplies the wrapped neighbour by exp(+-i k_a L_a).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The same source builds twice: complex fields (Bloch phases, k_z), and, with
 * ORACLE_REAL, real fields for problems whose phases are all real and k_z = 0. */
#ifdef ORACLE_REAL
typedef double cx;
#define CI 0.0
#define RE(x) (x)
#define IM(x) (0.0)
#else
typedef double complex cx;
#define CI I
#define RE(x) creal(x)
#define IM(x) cimag(x)
#endif

#define OG_MAXPOLE 3   /* undamped Lorentz poles per material (the silica model has three) */

typedef struct {
    int n[3];            /* cells along x, y, z; n[2] == 1 for a 2D cross-section */
    int twod;            /* 1: fields vary as exp(i kz z); d/dz -> i kz (Sec. III B) */
    int eact[3], hact[3];/* components that can be non-zero (TE/TM decouple exactly at k_z = 0) */
    double kz;
    double dx, dt, sigma;
    double bloch_re[3], bloch_im[3];   /* exp(i k_a L_a) for each axis (1 when not Bloch) */
    const double *ce[3];  /* 1/eps_inf at the E_c sites, 0 inside PEC */
    const double *ch[3];  /* 1/mu at the H_c sites, 0 inside PMC */
    int npole;            /* Lorentz poles per E site, 0..OG_MAXPOLE (0: non-dispersive everywhere) */
    const double *lde[OG_MAXPOLE][3]; /* Delta-eps_j of pole j at the E_c sites (0: no such pole there) */
    const double *lw0[OG_MAXPOLE][3]; /* omega_j of pole j at the E_c sites */
    /* CPML along axis a, per site index along that axis, [0] integer sites, [1] half sites */
    const double *pb[3][2], *pc[3][2], *pk[3][2];
    /* Cylindrical (r, z) cross-section with fields ~ exp(i m phi) (Sec. III C and the appendix on
     * cylindrical coordinates): axis 0 is r (r = 0 at i = 0, PEC wall at r = n[0] Delta), axis 1
     * is z; components 0, 1, 2 are (r, z, phi) on the sites of (x, y, z) above. */
    int cyl;
    double mphi;
} og_grid;

typedef struct {
    int magnetic;        /* 0: J source (sigma on D), 1: K source (sigma on B) */
    int nsteps;
    int nsrc;
    const int *src_comp, *src_idx;
    const double *src_re, *src_im;
    int nset;            /* number of surface functionals measured every step */
    const int *set_ptr;  /* CSR offsets, nset + 1 entries */
    const int *m_comp, *m_idx;
    const double *m_re, *m_im;
} og_sim;

static int idx3(const og_grid *g, int i, int j, int k) { return (k * g->n[1] + j) * g->n[0] + i; }

/* Forward difference along axis a of F at (i,j,k): (F(+1) - F(0)) / Delta, used
 * for the curl of E at H sites.  Wrap with the Bloch factor exp(+i k L). */
static cx dfwd(const og_grid *g, const cx *F, int a, int i, int j, int k)
{
    int c[3] = {i, j, k};
    cx here = F[idx3(g, i, j, k)];
    if (a == 2 && g->twod) return CI * g->kz * here;
    cx ph = 1.0;
    c[a] += 1;
    if (c[a] == g->n[a]) { c[a] = 0; ph = g->bloch_re[a] + CI * g->bloch_im[a]; }
    return (ph * F[idx3(g, c[0], c[1], c[2])] - here) / g->dx;
}

/* Backward difference along a: (F(0) - F(-1)) / Delta, used for the curl of H at E sites. */
static cx dbwd(const og_grid *g, const cx *F, int a, int i, int j, int k)
{
    int c[3] = {i, j, k};
    cx here = F[idx3(g, i, j, k)];
    if (a == 2 && g->twod) return CI * g->kz * here;
    cx ph = 1.0;
    c[a] -= 1;
    if (c[a] < 0) { c[a] = g->n[a] - 1; ph = g->bloch_re[a] - CI * g->bloch_im[a]; }
    return (here - ph * F[idx3(g, c[0], c[1], c[2])]) / g->dx;
}

/* One CPML-stretched derivative term: (1/kappa) dF + psi, psi <- b psi + c dF.
 * `half` selects the half-integer site profile along axis a. */
static cx stretch(const og_grid *g, int a, int half, int pos, cx d, cx *psi)
{
    if (a == 2 && g->twod) return d;
    if (!g->pb[a][half]) return d;
    double b = g->pb[a][half][pos], c = g->pc[a][half][pos], ik = g->pk[a][half][pos];
    *psi = b * (*psi) + c * d;
    return ik * d + *psi;
}

/* curl E at the H sites (forward differences, half-site CPML profiles). */
static void curl_e(const og_grid *g, cx *const E[3], cx *out[3], cx *psi[3][3])
{
    int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int m = idx3(g, i, j, k);
                int pos[3] = {i, j, k};
                /* (curl E)_x = dEz/dy - dEy/dz, etc. */
                for (int c = 0; c < 3; ++c) {
                    if (!g->hact[c]) continue;
                    int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
                    cx t1 = stretch(g, a1, 1, pos[a1], dfwd(g, E[a2], a1, i, j, k), &psi[c][a1][m]);
                    cx t2 = stretch(g, a2, 1, pos[a2], dfwd(g, E[a1], a2, i, j, k), &psi[c][a2][m]);
                    out[c][m] = t1 - t2;
                }
            }
}

/* curl H at the E sites (backward differences, integer-site CPML profiles). */
static void curl_h(const og_grid *g, cx *const H[3], cx *out[3], cx *psi[3][3])
{
    int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int m = idx3(g, i, j, k);
                int pos[3] = {i, j, k};
                for (int c = 0; c < 3; ++c) {
                    if (!g->eact[c]) continue;
                    int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
                    cx t1 = stretch(g, a1, 0, pos[a1], dbwd(g, H[a2], a1, i, j, k), &psi[c][a1][m]);
                    cx t2 = stretch(g, a2, 0, pos[a2], dbwd(g, H[a1], a2, i, j, k), &psi[c][a2][m]);
                    out[c][m] = t1 - t2;
                }
            }
}

/* Cylindrical curls.  With F ~ exp(i m phi):
 *   (curl F)_r   = (i m / r) F_z - dF_phi/dz
 *   (curl F)_phi = dF_r/dz - dF_z/dr
 *   (curl F)_z   = (1/r) d(r F_phi)/dr - (i m / r) F_r
 * Sites: E_r, H_z, H_phi at r = (i + 1/2) Delta; E_z, E_phi, H_r at r = i Delta.  Across the
 * outer wall (i + 1 = n[0]) E vanishes; inside the axis (i - 1 < 0) H is taken as zero.  On
 * the axis the z component follows Stokes over the disk of radius Delta/2:
 * (curl H)_z(0) = (Delta/2) H_phi(Delta/2) / ((Delta/8) Delta) = 4 H_phi(Delta/2) / Delta, the weight
 * of the axis site being the disk area over 2 pi Delta.
 * E_phi(0) and H_r(0) carry no weight (r = 0) and are masked by the caller, as is E_z(0) for
 * m != 0 (E_z ~ r^|m| near the axis). */
static cx zwrap(const og_grid *g, const cx *F, int i, int j, int dir)
{
    int jj = j + dir;
    cx ph = 1.0;
    if (jj == g->n[1]) { jj = 0; ph = g->bloch_re[1] + CI * g->bloch_im[1]; }
    if (jj < 0) { jj = g->n[1] - 1; ph = g->bloch_re[1] - CI * g->bloch_im[1]; }
    return ph * F[jj * g->n[0] + i];
}

static void curl_e_cyl(const og_grid *g, cx *const E[3], cx *out[3])
{
    int nr = g->n[0], nz = g->n[1];
    double d = g->dx;
    cx im = CI * g->mphi;
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nr; ++i) {
            int m = j * nr + i;
            double ri = i * d, rh = (i + 0.5) * d, rp = (i + 1) * d;
            cx ephi_r = i + 1 < nr ? E[2][m + 1] : 0.0;     /* E_phi at r_{i+1} */
            cx ez_r = i + 1 < nr ? E[1][m + 1] : 0.0;       /* E_z at r_{i+1} */
            /* H_r at (r_i, z_{j+1/2}) */
            out[0][m] = (i > 0 ? im / ri * E[1][m] : 0.0) - (zwrap(g, E[2], i, j, 1) - E[2][m]) / d;
            /* H_z at (r_{i+1/2}, z_j) */
            out[1][m] = (rp * ephi_r - ri * E[2][m]) / (rh * d) - im / rh * E[0][m];
            /* H_phi at (r_{i+1/2}, z_{j+1/2}) */
            out[2][m] = (zwrap(g, E[0], i, j, 1) - E[0][m]) / d - (ez_r - E[1][m]) / d;
        }
}

static void curl_h_cyl(const og_grid *g, cx *const H[3], cx *out[3])
{
    int nr = g->n[0], nz = g->n[1];
    double d = g->dx;
    cx im = CI * g->mphi;
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nr; ++i) {
            int m = j * nr + i;
            double ri = i * d, rh = (i + 0.5) * d, rl = (i - 0.5) * d;
            cx hphi_l = i > 0 ? H[2][m - 1] : 0.0;          /* H_phi at r_{i-1/2} */
            cx hz_l = i > 0 ? H[1][m - 1] : 0.0;            /* H_z at r_{i-1/2} */
            /* E_r at (r_{i+1/2}, z_j) */
            out[0][m] = im / rh * H[1][m] - (H[2][m] - zwrap(g, H[2], i, j, -1)) / d;
            /* E_z at (r_i, z_{j+1/2}) */
            if (i > 0)
                out[1][m] = (rh * H[2][m] - rl * hphi_l) / (ri * d) - im / ri * H[0][m];
            else
                out[1][m] = 4.0 * H[2][m] / d;
            /* E_phi at (r_i, z_j) */
            out[2][m] = (H[0][m] - zwrap(g, H[0], i, j, -1)) / d - (H[1][m] - hz_l) / d;
        }
}

/* Lorentz polarisation, one step of P_j'' + sigma P_j' + w_j^2 P_j = deps_j w_j^2 E for every pole j
 * (Eq. (9), or the sum of poles of the silica model, with omega^2 -> xi^2 + i sigma xi and no damping,
 * central differences).  `first` applies the start P_j(-dt) = P_j(+dt) (P and P' vanish at the impulse). */
static void lorentz_step(const og_grid *g, cx *P[][3], cx *Pm[][3], cx *const E[3], int first, int N)
{
    double dt = g->dt, s = g->sigma;
    for (int j = 0; j < g->npole; ++j)
        for (int c = 0; c < 3; ++c)
            for (int m = 0; m < N; ++m) {
                double de = g->lde[j][c][m];
                if (de == 0.0) continue;
                double w2 = g->lw0[j][c][m] * g->lw0[j][c][m];
                cx pn;
                if (first)
                    pn = 0.5 * ((2.0 - w2 * dt * dt) * P[j][c][m] + de * w2 * dt * dt * E[c][m]);
                else
                    pn = ((2.0 - w2 * dt * dt) * P[j][c][m] - (1.0 - 0.5 * s * dt) * Pm[j][c][m] +
                          de * w2 * dt * dt * E[c][m]) / (1.0 + 0.5 * s * dt);
                Pm[j][c][m] = P[j][c][m];
                P[j][c][m] = pn;
            }
}

/* E = (D - sum_j P_j) / eps_inf */
static void fields_e(const og_grid *g, cx *E[3], cx *const D[3], cx *P[][3], int N)
{
    for (int c = 0; c < 3; ++c)
        if (g->eact[c])
            for (int m = 0; m < N; ++m) {
                cx d = D[c][m];
                for (int j = 0; j < g->npole; ++j) d -= P[j][c][m];
                E[c][m] = g->ce[c][m] * d;
            }
}

static void fields_h(const og_grid *g, cx *H[3], cx *const B[3], int N)
{
    for (int c = 0; c < 3; ++c)
        if (g->hact[c])
            for (int m = 0; m < N; ++m) H[c][m] = g->ch[c][m] * B[c][m];
}

static void measure(const og_sim *s, cx *const F[3], int step, double *out_re, double *out_im)
{
    for (int q = 0; q < s->nset; ++q) {
        cx acc = 0.0;
        for (int e = s->set_ptr[q]; e < s->set_ptr[q + 1]; ++e)
            acc += (s->m_re[e] + CI * s->m_im[e]) * F[s->m_comp[e]][s->m_idx[e]];
        out_re[(size_t)q * s->nsteps + step] = RE(acc);
        out_im[(size_t)q * s->nsteps + step] = IM(acc);
    }
}

/* One zeroed pool for E H D B tmp (x3), P_j and P_j-prev (x3 per pole), psi_e psi_h (x9). */
static cx *alloc_fields(int N, cx *E[3], cx *H[3], cx *D[3], cx *B[3], cx *P[][3], cx *Pm[][3], cx *T[3],
                        cx *pe[3][3], cx *ph[3][3])
{
    cx *pool = calloc((size_t)N * (3 * 5 + 6 * OG_MAXPOLE + 2 * 9), sizeof(cx));
    if (!pool) return NULL;
    cx *p = pool;
    for (int c = 0; c < 3; ++c) { E[c] = p; p += N; H[c] = p; p += N; D[c] = p; p += N; B[c] = p; p += N;
                                  T[c] = p; p += N; }
    for (int j = 0; j < OG_MAXPOLE; ++j)
        for (int c = 0; c < 3; ++c) { P[j][c] = p; p += N; Pm[j][c] = p; p += N; }
    for (int c = 0; c < 3; ++c) for (int a = 0; a < 3; ++a) { pe[c][a] = p; p += N; ph[c][a] = p; p += N; }
    return pool;
}

/* Run one simulation; out_re/out_im receive nset x nsteps samples s(n), n = 1..T.
 * Returns 0 on success, -1 on allocation failure. */
int oracle_run(const og_grid *g, const og_sim *s, double *out_re, double *out_im)
{
    int N = g->n[0] * g->n[1] * g->n[2];
    cx *E[3], *H[3], *D[3], *B[3], *P[OG_MAXPOLE][3], *Pm[OG_MAXPOLE][3], *T[3], *pe[3][3], *ph[3][3];
    cx *pool = alloc_fields(N, E, H, D, B, P, Pm, T, pe, ph);
    if (!pool) return -1;

    double dt = g->dt, sg = g->sigma;
    double a_s = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);   /* conductive decay */
    double b_s = dt / (1.0 + 0.5 * sg * dt);

    /* Impulse J = delta(t) f (or K): the flux right after t = 0 is the source term. */
    cx **src = s->magnetic ? B : D;
    for (int e = 0; e < s->nsrc; ++e)
        src[s->src_comp[e]][s->src_idx[e]] += s->src_re[e] + CI * s->src_im[e];

    if (!s->magnetic) {
        fields_e(g, E, D, P, N);
        for (int n = 1; n <= s->nsteps; ++n) {
            /* B^{n-1/2} = B^{n-3/2} - dt curl E^{n-1}; the first step is a half step from B(0) = 0 */
            double h = (n == 1) ? 0.5 * dt : dt;
            if (g->cyl) curl_e_cyl(g, E, T); else curl_e(g, E, T, pe);
            for (int c = 0; c < 3; ++c) if (g->hact[c]) for (int m = 0; m < N; ++m) B[c][m] -= h * T[c][m];
            fields_h(g, H, B, N);
            /* P^n from E^{n-1} */
            lorentz_step(g, P, Pm, E, n == 1, N);
            /* D^n = a D^{n-1} + b curl H^{n-1/2}  (sigma on D) */
            if (g->cyl) curl_h_cyl(g, H, T); else curl_h(g, H, T, ph);
            for (int c = 0; c < 3; ++c) if (g->eact[c]) for (int m = 0; m < N; ++m) D[c][m] = a_s * D[c][m] + b_s * T[c][m];
            fields_e(g, E, D, P, N);
            measure(s, E, n - 1, out_re, out_im);
        }
    } else {
        fields_h(g, H, B, N);
        for (int n = 1; n <= s->nsteps; ++n) {
            double h = (n == 1) ? 0.5 * dt : dt;
            /* P^{n-1/2} from E^{n-3/2} (identically zero before the first D update) */
            lorentz_step(g, P, Pm, E, 0, N);
            /* D^{n-1/2} = D^{n-3/2} + dt curl H^{n-1}; half step first (no sigma on D) */
            if (g->cyl) curl_h_cyl(g, H, T); else curl_h(g, H, T, ph);
            for (int c = 0; c < 3; ++c) if (g->eact[c]) for (int m = 0; m < N; ++m) D[c][m] += h * T[c][m];
            fields_e(g, E, D, P, N);
            /* B^n = a B^{n-1} - b curl E^{n-1/2}  (sigma on B) */
            if (g->cyl) curl_e_cyl(g, E, T); else curl_e(g, E, T, pe);
            for (int c = 0; c < 3; ++c) if (g->hact[c]) for (int m = 0; m < N; ++m) B[c][m] = a_s * B[c][m] - b_s * T[c][m];
            fields_h(g, H, B, N);
            measure(s, H, n - 1, out_re, out_im);
        }
    }
    free(pool);
    return 0;
}

/* Free evolution from given initial fields (no source, no measurement), used by
 * the lattice pins: E^0 and B^{-1/2}-free start exactly as in oracle_run, then
 * `nsteps` full steps; the final E^T, H^{T-1/2} are written back.  D, B are the
 * flux fields (D = E / ce where ce != 0).  Electric ordering, sigma on D. */
int oracle_evolve(const og_grid *g, int nsteps, double *e_re, double *e_im, double *h_re, double *h_im,
                  double *hprev_re, double *hprev_im)
{
    int N = g->n[0] * g->n[1] * g->n[2];
    cx *E[3], *H[3], *D[3], *B[3], *P[OG_MAXPOLE][3], *Pm[OG_MAXPOLE][3], *T[3], *pe[3][3], *ph[3][3];
    cx *pool = alloc_fields(N, E, H, D, B, P, Pm, T, pe, ph);
    if (!pool) return -1;
    double dt = g->dt, sg = g->sigma;
    double a_s = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
    double b_s = dt / (1.0 + 0.5 * sg * dt);
    for (int c = 0; c < 3; ++c)
        for (int m = 0; m < N; ++m) {
            double ce = g->ce[c][m];
            D[c][m] = ce != 0.0 ? (e_re[c * N + m] + CI * e_im[c * N + m]) / ce : 0.0;
            double chv = g->ch[c][m];
            B[c][m] = chv != 0.0 ? (h_re[c * N + m] + CI * h_im[c * N + m]) / chv : 0.0;
        }
    fields_e(g, E, D, P, N);
    fields_h(g, H, B, N);
    int first = 1;
    for (int n = 1; n <= nsteps; ++n) {
        double h = first ? 0.5 * dt : dt;
        for (int c = 0; c < 3; ++c) for (int m = 0; m < N; ++m) { hprev_re[c * N + m] = RE(H[c][m]); hprev_im[c * N + m] = IM(H[c][m]); }
        if (g->cyl) curl_e_cyl(g, E, T); else curl_e(g, E, T, pe);
        for (int c = 0; c < 3; ++c) if (g->hact[c]) for (int m = 0; m < N; ++m) B[c][m] -= h * T[c][m];
        fields_h(g, H, B, N);
        if (g->cyl) curl_h_cyl(g, H, T); else curl_h(g, H, T, ph);
        for (int c = 0; c < 3; ++c) if (g->eact[c]) for (int m = 0; m < N; ++m) D[c][m] = a_s * D[c][m] + b_s * T[c][m];
        fields_e(g, E, D, P, N);
        first = 0;
    }
    for (int c = 0; c < 3; ++c)
        for (int m = 0; m < N; ++m) {
            e_re[c * N + m] = RE(E[c][m]); e_im[c * N + m] = IM(E[c][m]);
            h_re[c * N + m] = RE(H[c][m]); h_im[c * N + m] = IM(H[c][m]);
        }
    free(pool);
    return 0;
}
