// Internal plan representation shared by the host planner and the executor.
#pragma once
#include <cstdint>
#include <deque>
#include <string>
#include <vector>

#include "casimir.h"

namespace cas {

// A field array of a kernel family: which physical field (0 = E, 1 = H) and
// component it stores, where its sites sit (in cells), and the sign relating
// the stored value to the physical field.
struct ArraySpec {
    int field;
    int comp;
    double off[3];
    double sign;
};

enum Family { FAM_TM = 0, FAM_TE = 1, FAM_FULL = 2 };

// Kernel family layouts.
//  TM (2D, k_z = 0): u = E_z (i, j), vx = H_x (i, j+1/2), vy = H_y (i+1/2, j).
//  TE (2D, k_z = 0) uses the same update on the lattice shifted by half a cell
//  with u = H_z (i+1/2, j+1/2), vx = -E_x (i+1/2, j+1), vy = -E_y (i+1, j+1/2):
//  Maxwell's equations are invariant under E -> H, H -> -E, eps <-> mu.
//  FULL (2D with k_z, or 3D): Ex, Ey, Ez, Hx, Hy, Hz on the standard Yee sites.
int family_arrays(int family, ArraySpec out[6]);

struct Entry {
    int arr;          // array index within the family
    int64_t idx;      // flat site index (k*ny + j)*nx + i
    double re, im;    // value (source) or weight (measurement)
};

// One rasterised lattice: the coefficient of every array at every cell,
// deduplicated into a per-cell material id and a small table.
struct Geo {
    int family = 0;
    int kpt = 0;
    int n[3] = {1, 1, 1};
    int narr = 0;
    std::vector<uint8_t> mat;       // per cell
    std::vector<double> table;      // [id * narr + a]: 1/eps or 1/mu at that site, 0 masks PEC/PMC
    int nmat = 0;
    // Lorentz ADE (FULL family only): per E-array id and pole q -> (delta_eps, omega0)
    std::vector<double> lorentz;    // [(id * npoles + q) * 6 + 2*c + {0,1}] for c = 0..2
    int npoles = 0;                 // poles in use (present poles come first at every site)
    bool has_lorentz = false;
    double bloch_re[3] = {1, 1, 1}, bloch_im[3] = {0, 0, 0};
    double kz = 0.0;
    bool complex_fields = false;
    bool cyl = false;               // cylindrical (r, z) lattice, fields ~ exp(i m phi)
    int mphi = 0;
    // CPML per axis a and site kind h (0 integer, 1 half): b, c, 1/kappa along that axis
    std::vector<double> pml[3][2][3];
    bool has_pml[3] = {false, false, false};
};

struct Sim {
    int kpt, face, n1, n2;
    int kind;          // 0 = J (electric, sigma on D), 1 = K (magnetic, sigma on B)
    int comp;          // source component
    int family;
    int geo;           // index into PlanData::geos
    int second_u;      // TM/TE families: 1 if the measured (sigma) group is u, 0 if it is (vx, vy)
    std::vector<Entry> src;   // stored-field values right after the impulse
    std::vector<Entry> meas;  // s(n) = sum re * field (+ i im for complex fields)
};

struct PlanData {
    PlanData() = default;
    PlanData(const PlanData &) = delete;              // objects point into `masks`
    PlanData &operator=(const PlanData &) = delete;
    casimir_problem prob{};
    std::vector<casimir_object> objects;
    std::deque<std::vector<uint8_t>> masks;   // copies of the grid objects' masks (stable addresses)
    std::vector<casimir_face> faces;
    std::vector<casimir_kpoint> kpoints;
    double dx = 0, dt = 0;
    std::vector<Geo> geos;
    std::vector<Sim> sims;
    std::vector<double> gw;          // w_n = 2 dt Im g(-n dt), n = 1..T
    std::vector<double> kweight;     // per k-point
};

int build_plan(const casimir_problem *p, PlanData *out, std::string *err);

// Im g(-t) (plain kernel of Appendix A), independent of any oracle code.
double img_plain(double t, double sigma);

}  // namespace cas
