// Host-side planner: from a casimir_problem to rasterised lattices, face
// pixels, harmonic sources, measurement functionals and g(-t) weights.
//
// Method: McCauley et al., arXiv:0906.5170, Sec. II (force as a sum of
// harmonic-source simulations, Eqs. (1), (3)-(6)), Sec. III (cosine basis per
// face, Eq. (7); sources spread onto the Yee grid), Appendix A (g(t)).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <array>
#include <complex>
#include <thread>

#include "plan.h"

namespace cas {

namespace {
// Host threads for rasterising a lattice: the hardware's, at most 16; the environment
// variable CASIMIR_PLAN_THREADS (1..64) overrides the count.
int plan_threads()
{
    if (const char *e = std::getenv("CASIMIR_PLAN_THREADS")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 64) return v;
    }
    return (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
}

constexpr double kPi = 3.14159265358979323846;
constexpr double kTol = 1e-6;   // geometric tolerance, in cells

struct Mat {
    double eps, mu;
    bool pec, pmc;
    double de[CASIMIR_MAX_POLES], w0[CASIMIR_MAX_POLES];   // Lorentz poles, the present ones first
};

bool inside(const casimir_object &o, const double x[3], int dims, double d)
{
    double tol = kTol * d;
    if (o.shape == CASIMIR_SHAPE_BOX) {
        for (int a = 0; a < dims; ++a)
            if (x[a] < o.lo[a] - tol || x[a] > o.hi[a] + tol) return false;
        return true;
    }
    if (o.shape == CASIMIR_SHAPE_GRID) {
        // the union of the closed filled voxels: test the voxels within the tolerance of x
        // along each axis (one, or two when x lies on a voxel face)
        int c[3][2];
        for (int a = 0; a < 3; ++a) {
            if (a >= dims) { c[a][0] = c[a][1] = 0; continue; }
            if (x[a] < o.lo[a] - tol || x[a] > o.hi[a] + tol) return false;
            const double h = (o.hi[a] - o.lo[a]) / o.mask_n[a];
            const double u = (x[a] - o.lo[a]) / h, t = tol / h;
            c[a][0] = std::max(0, (int)std::floor(u - t));
            c[a][1] = std::min(o.mask_n[a] - 1, (int)std::floor(u + t));
        }
        for (int k = c[2][0]; k <= c[2][1]; ++k)
            for (int j = c[1][0]; j <= c[1][1]; ++j)
                for (int i = c[0][0]; i <= c[0][1]; ++i)
                    if (o.mask[((size_t)k * o.mask_n[1] + j) * o.mask_n[0] + i]) return true;
        return false;
    }
    double r2 = 0;
    for (int a = 0; a < dims; ++a) r2 += (x[a] - o.center[a]) * (x[a] - o.center[a]);
    return r2 <= (o.radius + tol) * (o.radius + tol);
}

Mat material_at(const PlanData &P, const double x[3])
{
    const casimir_problem &p = P.prob;
    Mat m{p.bg_eps, p.bg_mu, false, false, {}, {}};
    double d = P.dx;
    for (const auto &o : P.objects) {
        if (!inside(o, x, p.dims, d)) continue;
        m = Mat{p.bg_eps, p.bg_mu, false, false, {}, {}};
        switch (o.kind) {
        case CASIMIR_MAT_PEC: m.pec = true; break;
        case CASIMIR_MAT_PMC: m.pmc = true; break;
        case CASIMIR_MAT_DIELECTRIC: m.eps = o.eps; m.mu = o.mu; break;
        case CASIMIR_MAT_LORENTZ: {
            m.eps = o.eps_inf;
            m.mu = 1.0;
            int q = 0;
            for (int j = 0; j < CASIMIR_MAX_POLES; ++j)
                if (o.delta_eps[j] != 0.0) { m.de[q] = o.delta_eps[j]; m.w0[q] = o.omega0[j]; ++q; }
            break;
        }
        }
    }
    return m;
}

// Canonical coordinate of a site along axis a in [0, L).
double canon(double x, double L)
{
    if (x >= 0.0 && x <= L - 1e-9 * L) return x;   // already canonical (fmod would return x)
    double y = std::fmod(x, L);
    if (y < 0) y += L;
    if (y > L - 1e-9 * L) y = 0.0;
    return y;
}

void pml_profile(int n, int cells, double d, double dt, int half, std::vector<double> out[3])
{
    // Polynomial grading of order 3 with reflection 1e-8, kappa = 1, and a
    // frequency shift alpha falling linearly from 0.05 at the inner interface
    // to 0 at the wall (the paper gives no CPML parameters).
    double w = cells * d, L = n * d;
    double smax = -4.0 * std::log(1e-8) / (2.0 * w);
    for (int q = 0; q < 3; ++q) out[q].assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double x = (i + (half ? 0.5 : 0.0)) * d;
        double rho = std::max((w - x) / w, (x - (L - w)) / w);
        rho = std::min(1.0, std::max(0.0, rho));
        double sg = smax * rho * rho * rho;
        double kap = 1.0;
        double al = 0.05 * (1.0 - rho);
        double b = std::exp(-(sg / kap + al) * dt);
        double c = sg > 0 ? sg / (sg * kap + kap * kap * al) * (b - 1.0) : 0.0;
        out[0][i] = b;
        out[1][i] = c;
        out[2][i] = 1.0 / kap;
    }
}

struct Pix {
    std::vector<std::array<double, 3>> x;   // centres
    std::vector<int> t;                     // tangential axes
    std::vector<int> cnt;                   // pixels per tangential axis
    double dA;
};

Pix face_pixels(const PlanData &P, const casimir_face &f)
{
    Pix px;
    int dims = P.prob.dims;
    double d = P.dx;
    for (int b = 0; b < dims; ++b)
        if (b != f.axis) {
            px.t.push_back(b);
            px.cnt.push_back((int)std::lround((f.hi[b] - f.lo[b]) / d));
        }
    px.dA = std::pow(d, dims - 1);
    int n0 = px.cnt[0], n1 = px.cnt.size() > 1 ? px.cnt[1] : 1;
    for (int p = 0; p < n0; ++p)
        for (int q = 0; q < n1; ++q) {
            std::array<double, 3> c{0, 0, 0};
            c[f.axis] = f.pos;
            c[px.t[0]] = f.lo[px.t[0]] + (p + 0.5) * d;
            if (px.t.size() > 1) c[px.t[1]] = f.lo[px.t[1]] + (q + 0.5) * d;
            px.x.push_back(c);
        }
    return px;
}

// Cosine basis of Eq. (7) on a face, normalised on the pixel centres:
// f_0 = sqrt(1/L), f_n = sqrt(2/L) cos(n pi s / L); products in 3D.
double basis_value(const PlanData &P, const Pix &px, int pix, int n1, int n2)
{
    if (P.prob.basis == CASIMIR_BASIS_POINT) return pix == n1 ? 1.0 / std::sqrt(px.dA) : 0.0;
    double d = P.dx;
    int nn[2] = {n1, n2};
    int idx[2] = {px.cnt.size() > 1 ? pix / px.cnt[1] : pix, px.cnt.size() > 1 ? pix % px.cnt[1] : 0};
    double v = 1.0;
    for (size_t t = 0; t < px.t.size(); ++t) {
        double L = px.cnt[t] * d;
        double s = (idx[t] + 0.5) * d;
        v *= nn[t] == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L) * std::cos(nn[t] * kPi * s / L);
    }
    return v;
}

using cplx = std::complex<double>;

// Linear interpolation weights from the sites of array `as` to point x.
void stencil(const PlanData &P, const Geo &g, const ArraySpec &as, const double x[3],
             std::vector<std::pair<int64_t, cplx>> &out)
{
    out.clear();
    int dims = P.prob.dims;
    double d = P.dx;
    std::vector<std::pair<int, cplx>> ax[3];
    for (int a = 0; a < 3; ++a) {
        if (a >= dims) { ax[a].push_back({0, 1.0}); continue; }
        double u = x[a] / d - as.off[a];
        double fl = std::floor(u);
        double t = u - fl;
        long i0 = (long)fl;
        if (t < 1e-9) t = 0.0;
        else if (t > 1.0 - 1e-9) { i0 += 1; t = 0.0; }
        int n = g.n[a];
        cplx ph(g.bloch_re[a], g.bloch_im[a]);
        auto push = [&](long i, double w) {
            long q = (long)std::floor((double)i / n);
            cplx f = 1.0;
            for (long r = 0; r < std::labs(q); ++r) f *= (q > 0 ? ph : std::conj(ph));
            ax[a].push_back({(int)(i - q * n), w * f});
        };
        push(i0, 1.0 - t);
        if (t > 0.0) push(i0 + 1, t);
    }
    for (auto &ei : ax[0])
        for (auto &ej : ax[1])
            for (auto &ek : ax[2])
                out.push_back({((int64_t)ek.first * g.n[1] + ej.first) * g.n[0] + ei.first,
                               ei.second * ej.second * ek.second});
}

int find_array(int family, int field, int comp, const ArraySpec *arrs, int narr)
{
    for (int a = 0; a < narr; ++a)
        if (arrs[a].field == field && arrs[a].comp == comp) return a;
    (void)family;
    return -1;
}

// `same` (or null): a lattice of the same family (and, cylindrical, the same m) built for
// another k-point.  Materials, CPML and the Lorentz table do not depend on k, so they are
// copied from it instead of being rasterised again.
int build_geo(const PlanData &P, int family, int kpt, Geo *g, std::string *err, const Geo *same)
{
    const casimir_problem &p = P.prob;
    ArraySpec arrs[6];
    int narr = family_arrays(family, arrs);
    g->family = family;
    g->kpt = kpt;
    g->narr = narr;
    for (int a = 0; a < 3; ++a) g->n[a] = p.n[a];
    const double *k = P.kpoints[kpt].k;
    bool cplxf = false;
    for (int a = 0; a < p.dims; ++a) {
        if (p.bc[a] == CASIMIR_BC_PERIODIC) {
            double ph = k[a] * p.n[a] * P.dx;
            g->bloch_re[a] = std::cos(ph);
            g->bloch_im[a] = std::sin(ph);
            if (std::fabs(g->bloch_im[a]) > 0) cplxf = true;
        }
    }
    if (p.dims == 2) g->kz = k[2];
    const bool cyl = p.coords == CASIMIR_COORDS_CYLINDRICAL;
    if (cyl) {
        // r is not periodic: nothing couples across r = R (the PEC wall) or below the axis
        g->cyl = true;
        g->mphi = P.kpoints[kpt].m;
        g->kz = 0.0;
        g->bloch_re[0] = 0.0;
        g->bloch_im[0] = 0.0;
    }
    // a complex Bloch phase needs complex fields; k_z alone keeps them real (see the kernel)
    g->complex_fields = cplxf;
    if ((cplxf || g->kz != 0.0) && family != FAM_FULL) { *err = "k_z or a complex Bloch phase needs polarization FULL"; return CASIMIR_EINVAL; }

    if (same) {
        g->mat = same->mat;
        g->table = same->table;
        g->nmat = same->nmat;
        g->lorentz = same->lorentz;
        g->npoles = same->npoles;
        g->has_lorentz = same->has_lorentz;
        for (int a = 0; a < 3; ++a) {
            g->has_pml[a] = same->has_pml[a];
            for (int h = 0; h < 2; ++h)
                for (int q = 0; q < 3; ++q) g->pml[a][h][q] = same->pml[a][h][q];
        }
        return CASIMIR_OK;
    }
    int64_t ncell = (int64_t)p.n[0] * p.n[1] * p.n[2];
    g->mat.assign(ncell, 0);
    constexpr int NPK = 6 * CASIMIR_MAX_POLES;   // (delta_eps, omega0) per pole and E component
    double L[3] = {p.n[0] * P.dx, p.n[1] * P.dx, p.n[2] * P.dx};
    // key of cell (i, j, kk): every array's coefficient, then every E component's poles
    auto cell_key = [&](int i, int j, int kk, std::vector<double> &key) {
        std::fill(key.begin(), key.end(), 0.0);
        for (int a = 0; a < narr; ++a) {
            const ArraySpec &as = arrs[a];
            double x[3] = {(i + as.off[0]) * P.dx, (j + as.off[1]) * P.dx, (kk + as.off[2]) * P.dx};
            bool wall = false;
            for (int ax = 0; ax < p.dims; ++ax) {
                x[ax] = canon(x[ax], L[ax]);
                if (cyl && ax == 0) continue;   // r = 0 is the axis, the wall r = R lies beyond the grid
                if (as.field == 0 && (p.bc[ax] == CASIMIR_BC_PEC || p.bc[ax] == CASIMIR_BC_PML) &&
                    std::fabs(x[ax]) < kTol * P.dx)
                    wall = true;
            }
            // on the axis: E_phi and H_r carry no weight (r = 0); E_z ~ r^|m| vanishes for m != 0
            bool axis_mask = cyl && i == 0 && as.off[0] == 0.0 &&
                             ((as.field == 0 && as.comp == 2) || (as.field == 1 && as.comp == 0) ||
                              (as.field == 0 && as.comp == 1 && g->mphi != 0));
            Mat m = material_at(P, x);
            double c;
            if (axis_mask) {
                c = 0.0;
            } else if (as.field == 0) {
                c = (m.pec || wall) ? 0.0 : 1.0 / m.eps;
                if (!(m.pec || wall))
                    for (int q = 0; q < CASIMIR_MAX_POLES && m.de[q] != 0.0; ++q) {
                        key[narr + 6 * q + 2 * as.comp] = m.de[q];
                        key[narr + 6 * q + 2 * as.comp + 1] = m.w0[q];
                    }
            } else {
                c = m.pmc ? 0.0 : 1.0 / m.mu;
            }
            key[a] = c;
        }
    };
    // Material ids in order of first occurrence in the scan (x fastest).  Ranges of rows are
    // numbered in parallel, each in its own first-seen order; merging the ranges in scan order
    // then gives every key the id a single pass would give it.
    const int64_t rows = (int64_t)p.n[1] * p.n[2];
    const int nchunk = (int)std::min<int64_t>(ncell >= (1 << 16) ? plan_threads() : 1, rows);
    std::vector<std::vector<std::vector<double>>> chunk_keys(nchunk);
    std::vector<char> overflow(nchunk, 0), failed(nchunk, 0);
    auto number_rows_range = [&](int s) {
        std::map<std::vector<double>, int> local;
        std::vector<double> key(narr + NPK), prev_key;
        int prev_id = -1;
        for (int64_t r = rows * s / nchunk; r < rows * (s + 1) / nchunk; ++r) {
            const int kk = (int)(r / p.n[1]), j = (int)(r % p.n[1]);
            for (int i = 0; i < p.n[0]; ++i) {
                cell_key(i, j, kk, key);
                // neighbouring cells mostly share their key: try the previous cell's first
                int id;
                if (prev_id >= 0 && key == prev_key) {
                    id = prev_id;
                } else {
                    auto it = local.find(key);
                    if (it == local.end()) {
                        id = (int)local.size();
                        if (id > 255) { overflow[s] = 1; return; }   // the whole grid has more too
                        local.emplace(key, id);
                        chunk_keys[s].push_back(key);
                    } else {
                        id = it->second;
                    }
                    prev_key = key;
                    prev_id = id;
                }
                g->mat[r * p.n[0] + i] = (uint8_t)id;
            }
        }
    };
    auto number_rows = [&](int s) {
        // runs on a worker thread: nothing may escape it (an exception leaving a thread's
        // function terminates the process), so an allocation failure is flagged per range
        try {
            number_rows_range(s);
        } catch (...) {
            failed[s] = 1;
        }
    };
    {
        // ranges whose thread cannot be started are numbered on the calling thread
        std::vector<std::thread> pool;
        std::vector<int> inline_ranges{0};
        for (int s = 1; s < nchunk; ++s) {
            try {
                pool.emplace_back(number_rows, s);
            } catch (...) {
                inline_ranges.push_back(s);
            }
        }
        for (int s : inline_ranges) number_rows(s);
        for (auto &t : pool) t.join();
    }
    for (int s = 0; s < nchunk; ++s)
        if (failed[s]) { *err = "out of host memory while numbering material sites"; return CASIMIR_ENOMEM; }
    std::map<std::vector<double>, int> ids;
    for (int s = 0; s < nchunk; ++s) {
        if (overflow[s]) { *err = "more than 256 distinct material sites"; return CASIMIR_EINVAL; }
        uint8_t remap[256];
        for (size_t q = 0; q < chunk_keys[s].size(); ++q) {
            auto it = ids.find(chunk_keys[s][q]);
            if (it == ids.end()) {
                const int id = (int)ids.size();
                if (id > 255) {
                    *err = "more than 256 distinct material sites (found when merging the row ranges)";
                    return CASIMIR_EINVAL;
                }
                it = ids.emplace(chunk_keys[s][q], id).first;
            }
            remap[q] = (uint8_t)it->second;
        }
        for (int64_t c = rows * s / nchunk * p.n[0]; c < rows * (s + 1) / nchunk * p.n[0]; ++c) g->mat[c] = remap[g->mat[c]];
    }
    g->nmat = (int)ids.size();
    g->table.assign((size_t)g->nmat * narr, 0.0);
    // poles in use: the highest pole present at any site
    g->npoles = 0;
    for (auto &kv : ids)
        for (int q = 0; q < CASIMIR_MAX_POLES; ++q)
            for (int c = 0; c < 3; ++c)
                if (kv.first[narr + 6 * q + 2 * c] != 0.0) g->npoles = std::max(g->npoles, q + 1);
    g->has_lorentz = g->npoles > 0;
    g->lorentz.assign((size_t)g->nmat * 6 * g->npoles, 0.0);
    for (auto &kv : ids) {
        for (int a = 0; a < narr; ++a) g->table[(size_t)kv.second * narr + a] = kv.first[a];
        for (int q = 0; q < 6 * g->npoles; ++q) g->lorentz[(size_t)kv.second * 6 * g->npoles + q] = kv.first[narr + q];
    }
    for (int a = 0; a < p.dims; ++a)
        if (p.bc[a] == CASIMIR_BC_PML) {
            g->has_pml[a] = true;
            for (int h = 0; h < 2; ++h) pml_profile(p.n[a], p.pml_cells[a], P.dx, P.dt, h, g->pml[a][h]);
        }
    return CASIMIR_OK;
}

}  // namespace

int family_arrays(int family, ArraySpec out[6])
{
    if (family == FAM_TM) {
        out[0] = ArraySpec{0, 2, {0.0, 0.0, 0.5}, 1.0};
        out[1] = ArraySpec{1, 0, {0.0, 0.5, 0.5}, 1.0};
        out[2] = ArraySpec{1, 1, {0.5, 0.0, 0.5}, 1.0};
        return 3;
    }
    if (family == FAM_TE) {
        out[0] = ArraySpec{1, 2, {0.5, 0.5, 0.0}, 1.0};
        out[1] = ArraySpec{0, 0, {0.5, 1.0, 0.0}, -1.0};
        out[2] = ArraySpec{0, 1, {1.0, 0.5, 0.0}, -1.0};
        return 3;
    }
    out[0] = ArraySpec{0, 0, {0.5, 0.0, 0.0}, 1.0};
    out[1] = ArraySpec{0, 1, {0.0, 0.5, 0.0}, 1.0};
    out[2] = ArraySpec{0, 2, {0.0, 0.0, 0.5}, 1.0};
    out[3] = ArraySpec{1, 0, {0.0, 0.5, 0.5}, 1.0};
    out[4] = ArraySpec{1, 1, {0.5, 0.0, 0.5}, 1.0};
    out[5] = ArraySpec{1, 2, {0.5, 0.5, 0.0}, 1.0};
    return 6;
}

// Im g(-t) of Appendix A.  Rotating g(-t) = (1/2pi) int_0^inf g(xi) e^{i xi t} dxi
// onto xi = i eta gives the Laplace integral
//   Im g(-t) = (1/2pi) int_0^inf sqrt(1 + sigma/eta) (eta + sigma/2) e^{-eta t} d eta,
// evaluated with eta = e(tau) / t, e(tau) = exp(pi/2 sinh(tau)) (exp-sinh quadrature,
// which absorbs the eta^{-1/2} end point and the exponential tail; scaling by 1/t puts the
// integrand's peak near tau = 0).  With that scaling e^{-eta t} = e^{-e(tau)} does not depend
// on t, so the nodes e_k and the t-free part of their weights, e_k (pi/2) cosh(tau_k) e^{-e_k},
// are computed once and every t costs one square root per node.
namespace {
struct ExpSinhNodes {
    static constexpr double h = 1.0 / 64.0;
    std::vector<double> e, a;
    ExpSinhNodes()
    {
        for (int k = -6 * 64; k <= 6 * 64; ++k) {
            const double tau = k * h;
            const double ek = std::exp(0.5 * kPi * std::sinh(tau));
            const double ak = ek * 0.5 * kPi * std::cosh(tau) * std::exp(-ek);
            if (!(ek > 0.0) || !std::isfinite(ek) || !std::isfinite(ak)) continue;
            e.push_back(ek);
            a.push_back(ak);
        }
    }
};
}  // namespace

double img_plain(double t, double sigma)
{
    if (sigma == 0.0) return 1.0 / (2.0 * kPi * t * t);
    static const ExpSinhNodes nodes;
    const double st = sigma * t, hs = 0.5 * sigma, it = 1.0 / t;
    double sum = 0.0;
    for (size_t k = 0; k < nodes.e.size(); ++k) {
        const double ek = nodes.e[k];
        const double v = nodes.a[k] * std::sqrt(1.0 + st / ek) * (ek * it + hs);
        if (std::isfinite(v)) sum += v;
    }
    return sum * it * ExpSinhNodes::h / (2.0 * kPi);
}

int build_plan(const casimir_problem *pin, PlanData *P, std::string *err)
{
    const casimir_problem &p = *pin;
    if (p.dims != 2 && p.dims != 3) { *err = "dims must be 2 or 3"; return CASIMIR_EINVAL; }
    for (int a = 0; a < 3; ++a)
        if (p.n[a] < 1) { *err = "grid sizes must be >= 1"; return CASIMIR_EINVAL; }
    if (p.dims == 2 && p.n[2] != 1) { *err = "two-dimensional problems have n[2] == 1"; return CASIMIR_EINVAL; }
    if (!(p.resolution > 0) || !(p.courant > 0) || p.n_steps < 1 || !(p.sigma >= 0)) {
        *err = "resolution, courant, n_steps must be positive and sigma >= 0";
        return CASIMIR_EINVAL;
    }
    if (p.courant * std::sqrt((double)p.dims) >= 1.0) { *err = "courant number above the Yee stability limit"; return CASIMIR_EINVAL; }
    if (p.n_faces < 1 || !p.faces) { *err = "no stress-surface faces"; return CASIMIR_EINVAL; }
    if (p.n_kpoints < 1 || !p.kpoints) { *err = "no k-points"; return CASIMIR_EINVAL; }
    if (p.n_objects < 0 || (p.n_objects > 0 && !p.objects)) { *err = "objects"; return CASIMIR_EINVAL; }
    if (p.force_axis < 0 || p.force_axis >= p.dims) { *err = "force_axis"; return CASIMIR_EINVAL; }
    if (p.n_harm < 1) { *err = "n_harm must be >= 1"; return CASIMIR_EINVAL; }
    if (p.precision != CASIMIR_FP32 && p.precision != CASIMIR_FP64) { *err = "precision"; return CASIMIR_EINVAL; }
    if (p.g_variant != CASIMIR_G_PLAIN && p.g_variant != CASIMIR_G_ZINV) { *err = "g_variant"; return CASIMIR_EINVAL; }
    bool twod_pol = p.polarization == CASIMIR_POL_TM || p.polarization == CASIMIR_POL_TE || p.polarization == CASIMIR_POL_TETM;
    if (!twod_pol && p.polarization != CASIMIR_POL_FULL) { *err = "polarization"; return CASIMIR_EINVAL; }
    if (twod_pol && p.dims != 2) { *err = "TM/TE polarizations are two-dimensional"; return CASIMIR_EINVAL; }
    for (int a = 0; a < p.dims; ++a) {
        if (p.bc[a] < 0 || p.bc[a] > 2) { *err = "bc"; return CASIMIR_EINVAL; }
        if (p.bc[a] == CASIMIR_BC_PML && (p.pml_cells[a] < 1 || 2 * p.pml_cells[a] >= p.n[a])) {
            *err = "pml_cells";
            return CASIMIR_EINVAL;
        }
    }
    P->prob = p;
    P->objects.assign(p.objects, p.objects + p.n_objects);
    P->faces.assign(p.faces, p.faces + p.n_faces);
    P->kpoints.assign(p.kpoints, p.kpoints + p.n_kpoints);
    P->prob.objects = P->objects.data();
    P->prob.faces = P->faces.data();
    P->prob.kpoints = P->kpoints.data();
    P->dx = 1.0 / p.resolution;
    P->dt = p.courant * P->dx;
    for (auto &o : P->objects) {
        if (o.kind < 0 || o.kind > 3 || o.shape < 0 || o.shape > 2) { *err = "object kind/shape"; return CASIMIR_EINVAL; }
        if (o.shape == CASIMIR_SHAPE_GRID) {
            if (!o.mask) { *err = "grid object without a mask"; return CASIMIR_EINVAL; }
            for (int a = 0; a < 3; ++a)
                if (o.mask_n[a] < 1 || (a < p.dims && !(o.hi[a] > o.lo[a])) || (a >= p.dims && o.mask_n[a] != 1)) {
                    *err = "grid object: mask_n >= 1 and hi > lo on every used axis (mask_n[2] == 1 in 2D)";
                    return CASIMIR_EINVAL;
                }
            // the plan keeps its own copy of the mask
            P->masks.emplace_back(o.mask, o.mask + (size_t)o.mask_n[0] * o.mask_n[1] * o.mask_n[2]);
            o.mask = P->masks.back().data();
        } else {
            o.mask = nullptr;
        }
        if (o.kind == CASIMIR_MAT_DIELECTRIC && !(o.eps > 0 && o.mu > 0)) { *err = "dielectric eps, mu must be > 0"; return CASIMIR_EINVAL; }
        if (o.kind == CASIMIR_MAT_LORENTZ) {
            if (!(o.eps_inf > 0)) { *err = "lorentz eps_inf must be > 0"; return CASIMIR_EINVAL; }
            for (int j = 0; j < CASIMIR_MAX_POLES; ++j)
                if (!(o.delta_eps[j] >= 0) || (o.delta_eps[j] > 0 && !(o.omega0[j] > 0))) {
                    *err = "lorentz poles need delta_eps >= 0 and omega0 > 0";
                    return CASIMIR_EINVAL;
                }
        }
    }
    if (!(p.bg_eps > 0 && p.bg_mu > 0)) { *err = "background eps, mu must be > 0"; return CASIMIR_EINVAL; }
    for (auto &f : P->faces) {
        if (f.axis < 0 || f.axis >= p.dims || (f.sign != 1 && f.sign != -1)) { *err = "face axis/sign"; return CASIMIR_EINVAL; }
        for (int b = 0; b < p.dims; ++b) {
            if (b == f.axis) continue;
            double c = (f.hi[b] - f.lo[b]) / P->dx;
            if (c < 0.5 || std::fabs(c - std::lround(c)) > 1e-6) { *err = "face extents must be whole cells"; return CASIMIR_EINVAL; }
        }
    }

    if (p.coords != CASIMIR_COORDS_CARTESIAN && p.coords != CASIMIR_COORDS_CYLINDRICAL) { *err = "coords"; return CASIMIR_EINVAL; }
    if (p.coords == CASIMIR_COORDS_CYLINDRICAL) {
        if (p.dims != 2 || p.polarization != CASIMIR_POL_FULL || p.bc[0] != CASIMIR_BC_PEC) {
            *err = "cylindrical problems are (r, z) cross-sections with polarization FULL and a PEC wall at r = R";
            return CASIMIR_EINVAL;
        }
        if (p.bc[1] == CASIMIR_BC_PML) { *err = "cylindrical problems take PEC or periodic z boundaries"; return CASIMIR_EINVAL; }
        for (auto &o : P->objects)
            if (o.kind == CASIMIR_MAT_LORENTZ) { *err = "cylindrical problems take no Lorentz media"; return CASIMIR_EINVAL; }
        for (auto &k : P->kpoints) {
            if (k.k[0] != 0.0 || k.k[1] != 0.0 || k.k[2] != 0.0) { *err = "cylindrical k-points carry m only (k = 0)"; return CASIMIR_EINVAL; }
            // the i m / r terms next to the axis bound the step: the spatial operator's largest
            // eigenvalue is below max(9, 8 + 4 m^2) / Delta^2
            double lam = std::max(9.0, 8.0 + 4.0 * (double)k.m * (double)k.m);
            if (p.courant * p.courant * lam >= 4.0) { *err = "courant number above the cylindrical stability limit for this m"; return CASIMIR_EINVAL; }
        }
    }
    if (twod_pol) {
        for (auto &o : P->objects)
            if (o.kind == CASIMIR_MAT_LORENTZ) { *err = "Lorentz media need polarization FULL"; return CASIMIR_EINVAL; }
        for (int a = 0; a < p.dims; ++a)
            if (p.bc[a] == CASIMIR_BC_PML) { *err = "PML boundaries need polarization FULL"; return CASIMIR_EINVAL; }
    }
    // with d/dz -> i k_z the leapfrog is stable only for (dt/2)^2 (dims (2/dx)^2 + k_z^2) < 1
    if (p.dims == 2)
        for (auto &k : P->kpoints) {
            double lim = 0.25 * P->dt * P->dt * (2.0 * 4.0 / (P->dx * P->dx) + k.k[2] * k.k[2]);
            if (lim >= 1.0) { *err = "k_z beyond the time-step stability limit"; return CASIMIR_EINVAL; }
        }
    // Dispersive media: the lattice dispersion relation Omega^2 eps(Omega^2) = k^2, with
    // Omega = (2/dt) sin(omega dt / 2), has every root Omega^2 below X = 4/dt^2 (omega real)
    // exactly when each pole has omega_j dt < 2 and X eps(X) exceeds the largest lattice k^2
    // (x eps(x) increases on every branch between poles), i.e. eps(X) > (dt/2)^2 k_max^2.
    {
        double q = 3.0 * p.courant * p.courant;   // 3D: (dt/2)^2 * 12 / dx^2
        if (p.dims == 2) {
            q = 0.0;
            for (auto &k : P->kpoints)
                q = std::max(q, 0.25 * P->dt * P->dt * (8.0 / (P->dx * P->dx) + k.k[2] * k.k[2]));
        }
        for (auto &o : P->objects) {
            if (o.kind != CASIMIR_MAT_LORENTZ) continue;
            double epsX = o.eps_inf;
            for (int j = 0; j < CASIMIR_MAX_POLES; ++j) {
                if (o.delta_eps[j] == 0.0) continue;
                const double wd2 = o.omega0[j] * o.omega0[j] * P->dt * P->dt;
                if (wd2 >= 4.0) { *err = "lorentz pole with omega0 dt >= 2 (unstable)"; return CASIMIR_EINVAL; }
                epsX -= o.delta_eps[j] * wd2 / (4.0 - wd2);
            }
            if (epsX <= q) { *err = "lorentz medium unstable at this time step (eps(4/dt^2) below the lattice bound)"; return CASIMIR_EINVAL; }
        }
    }
    // families
    std::vector<int> fams;
    if (p.polarization == CASIMIR_POL_TM || p.polarization == CASIMIR_POL_TETM) fams.push_back(FAM_TM);
    if (p.polarization == CASIMIR_POL_TE || p.polarization == CASIMIR_POL_TETM) fams.push_back(FAM_TE);
    if (p.polarization == CASIMIR_POL_FULL) fams.push_back(FAM_FULL);

    // g weights, Eq. (1) by the rectangle rule at t_n = n dt
    int T = p.n_steps;
    P->gw.resize(T);
    for (int n = 1; n <= T; ++n) {
        double t = n * P->dt, im;
        if (p.g_variant == CASIMIR_G_PLAIN) {
            im = img_plain(t, p.sigma);
        } else {
            // z-invariant PEC/vacuum kernel: the extra factor i*omega/2 of the text of
            // Appendix A.2, i.e. half of the closed form printed there.
            double s = p.sigma;
            im = 0.5 * (2.0 / (t * t * t) + 1.5 * s / (t * t) + 0.5 * s * s / t) / (2.0 * kPi);
        }
        P->gw[n - 1] = 2.0 * P->dt * im;
    }
    P->kweight.resize(p.n_kpoints);
    for (int k = 0; k < p.n_kpoints; ++k) P->kweight[k] = P->kpoints[k].weight;

    // lattices
    std::map<std::pair<int, int>, int> geo_of;
    std::map<std::pair<int, int>, int> lattice_of;   // (family, m if cylindrical) -> first geo built
    const bool cyl_coords = p.coords == CASIMIR_COORDS_CYLINDRICAL;
    for (int k = 0; k < p.n_kpoints; ++k)
        for (int fam : fams) {
            Geo g;
            const std::pair<int, int> lk{fam, cyl_coords ? P->kpoints[k].m : 0};
            auto li = lattice_of.find(lk);
            int rc = build_geo(*P, fam, k, &g, err, li == lattice_of.end() ? nullptr : &P->geos[li->second]);
            if (li == lattice_of.end()) lattice_of[lk] = (int)P->geos.size();
            if (rc) return rc;
            geo_of[{k, fam}] = (int)P->geos.size();
            P->geos.push_back(std::move(g));
        }

    // simulations: (k-point, face, harmonic, family, source kind, component)
    struct Src { int fam, kind, comp; };
    std::vector<Src> srcs;
    for (int fam : fams) {
        if (fam == FAM_TM) { srcs.push_back({fam, 0, 2}); srcs.push_back({fam, 1, 0}); srcs.push_back({fam, 1, 1}); }
        if (fam == FAM_TE) { srcs.push_back({fam, 0, 0}); srcs.push_back({fam, 0, 1}); srcs.push_back({fam, 1, 2}); }
        if (fam == FAM_FULL)
            for (int kind = 0; kind < 2; ++kind)
                for (int c = 0; c < 3; ++c) srcs.push_back({fam, kind, c});
    }
    using Stencil = std::vector<std::pair<int64_t, cplx>>;
    for (int k = 0; k < p.n_kpoints; ++k)
        for (int fi = 0; fi < p.n_faces; ++fi) {
            const casimir_face &f = P->faces[fi];
            Pix px = face_pixels(*P, f);
            std::vector<std::pair<int, int>> harms;
            if (p.basis == CASIMIR_BASIS_POINT) {
                for (size_t q = 0; q < px.x.size(); ++q) harms.push_back({(int)q, 0});
            } else {
                int h0 = std::min(p.n_harm, px.cnt[0]);
                int h1 = px.cnt.size() > 1 ? std::min(p.n_harm, px.cnt[1]) : 1;
                for (int a = 0; a < h0; ++a)
                    for (int b = 0; b < h1; ++b) harms.push_back({a, b});
            }
            // surface eps / mu at the pixels (Minkowski weight)
            std::vector<double> epsS(px.x.size()), muS(px.x.size());
            for (size_t q = 0; q < px.x.size(); ++q) {
                Mat m = material_at(*P, px.x[q].data());
                epsS[q] = m.eps;
                muS[q] = m.mu;
            }
            // interpolation stencils of every pixel onto the sites of one array of one family's
            // lattice at this k-point, shared by every harmonic and source of the face; each
            // stencil site also carries its index among the distinct sites the face touches
            struct Stencils {
                std::vector<Stencil> st;
                std::vector<std::vector<int>> uid;
                int nu = 0;
            };
            std::map<std::pair<int, int>, Stencils> stc;
            auto stencils = [&](int fam, const Geo &g, const ArraySpec &as, int arr) -> const Stencils & {
                auto it = stc.find({fam, arr});
                if (it != stc.end()) return it->second;
                Stencils &v = stc[{fam, arr}];
                v.st.resize(px.x.size());
                v.uid.resize(px.x.size());
                std::map<int64_t, int> sites;
                for (size_t q = 0; q < px.x.size(); ++q) {
                    stencil(*P, g, as, px.x[q].data(), v.st[q]);
                    for (auto &e : v.st[q]) v.uid[q].push_back(sites.emplace(e.first, (int)sites.size()).first->second);
                }
                v.nu = (int)sites.size();
                return v;
            };
            // entries of one simulation, summed per (array, site) and kept in first-touch order
            std::vector<int> slot[6];
            auto add = [&](std::vector<Entry> &v, int arr, int nu, int u, int64_t idx, cplx val) {
                std::vector<int> &sl = slot[arr];
                if ((int)sl.size() < nu) sl.resize(nu, -1);
                if (sl[u] < 0) {
                    sl[u] = (int)v.size();
                    v.push_back(Entry{arr, idx, val.real(), val.imag()});
                } else {
                    v[sl[u]].re += val.real();
                    v[sl[u]].im += val.imag();
                }
            };
            auto clear_slots = [&](const std::vector<Entry> &v, const std::vector<int> &u_of) {
                for (size_t e = 0; e < v.size(); ++e) slot[v[e].arr][u_of[e]] = -1;
            };
            std::vector<int> u_of;
            std::vector<double> fv(px.x.size());
            for (auto hm : harms) {
                for (size_t q = 0; q < px.x.size(); ++q) fv[q] = basis_value(*P, px, (int)q, hm.first, hm.second);
                for (auto s : srcs) {
                    // exact pruning: for force axis i and a face with normal a != i only c == a contributes
                    if (!(f.axis == p.force_axis || s.comp == f.axis)) continue;
                    Sim sim;
                    sim.kpt = k;
                    sim.face = fi;
                    sim.n1 = hm.first;
                    sim.n2 = hm.second;
                    sim.kind = s.kind;
                    sim.comp = s.comp;
                    sim.family = s.fam;
                    sim.geo = geo_of[{k, s.fam}];
                    const Geo &g = P->geos[sim.geo];
                    ArraySpec arrs[6];
                    int narr = family_arrays(s.fam, arrs);
                    int sa = find_array(s.fam, s.kind, s.comp, arrs, narr);
                    sim.second_u = (sa == 0) ? 1 : 0;
                    // source: flux after the impulse D_c = -(dA/dV) W_c^H f, stored as E = D/eps (masked)
                    const Stencils &ss = stencils(s.fam, g, arrs[sa], sa);
                    u_of.clear();
                    for (size_t q = 0; q < px.x.size(); ++q) {
                        if (fv[q] == 0.0) continue;
                        for (size_t j = 0; j < ss.st[q].size(); ++j) {
                            const auto &e = ss.st[q][j];
                            // cylindrical: the surface current on the surface of revolution averaged over
                            // the site's ring carries r(pixel) / w(site), w = r_site (Delta/8 on the axis)
                            double scale = 1.0;
                            if (g.cyl) {
                                double rs = ((double)(e.first % p.n[0]) + arrs[sa].off[0]) * P->dx;
                                scale = px.x[q][0] / (rs > 0.5 * kTol * P->dx ? rs : 0.125 * P->dx);
                            }
                            const size_t before = sim.src.size();
                            add(sim.src, sa, ss.nu, ss.uid[q][j], e.first, -std::conj(e.second) * fv[q] * scale / P->dx);
                            if (sim.src.size() > before) u_of.push_back(ss.uid[q][j]);
                        }
                    }
                    clear_slots(sim.src, u_of);
                    for (auto &e : sim.src) {
                        double c = g.table[(size_t)g.mat[e.idx] * narr + sa] * arrs[sa].sign;
                        e.re *= c;
                        e.im *= c;
                    }
                    // measurement: s_i = sum_k dA w_S f(x_k) [n_c F_i(x_k) - 1/2 n_i F_c(x_k)]
                    double nv[3] = {0, 0, 0};
                    nv[f.axis] = f.sign;
                    int i = p.force_axis;
                    u_of.clear();
                    for (size_t q = 0; q < px.x.size(); ++q) {
                        if (fv[q] == 0.0) continue;
                        double base = px.dA * (s.kind == 0 ? epsS[q] : muS[q]) * fv[q];
                        int comps[2] = {i, s.comp};
                        double coefs[2] = {nv[s.comp], -0.5 * nv[i]};
                        for (int t = 0; t < 2; ++t) {
                            if (coefs[t] == 0.0) continue;
                            int ma = find_array(s.fam, s.kind, comps[t], arrs, narr);
                            if (ma < 0) continue;   // component absent in this family: identically zero
                            const Stencils &sm = stencils(s.fam, g, arrs[ma], ma);
                            for (size_t j = 0; j < sm.st[q].size(); ++j) {
                                const size_t before = sim.meas.size();
                                add(sim.meas, ma, sm.nu, sm.uid[q][j], sm.st[q][j].first,
                                    sm.st[q][j].second * (base * coefs[t] * arrs[ma].sign));
                                if (sim.meas.size() > before) u_of.push_back(sm.uid[q][j]);
                            }
                        }
                    }
                    clear_slots(sim.meas, u_of);
                    P->sims.push_back(std::move(sim));
                }
            }
        }
    if (P->sims.empty()) { *err = "no contributing simulations"; return CASIMIR_EINVAL; }
    return CASIMIR_OK;
}

}  // namespace cas
