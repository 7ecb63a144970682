// sphere.cu -- the explicit MHD stage on a cubed-sphere shell (FP64): six
// equiangular patches of N x N angular cells times Nr radial cells between
// r_in and r_out, reflecting radial walls, the well-balanced deviation form
// under radial gravity, Contact-CT on the magnetic fluxes of the faces.
//
// The paper runs hydrodynamics on its cubed-sphere grid (Sect. 2.3) and MHD
// on its other grids; MHD here is the same scheme carried to this grid:
//   - The shell is a hexahedral mesh whose every cell, face and edge is an
//     angular entity (a cell, a side or a vertex of the spherical quad mesh
//     of the six patches, built once on the host) times a radial index.  A
//     side or vertex on a patch seam is one entity, shared by the patches
//     that meet there, so a seam face's flux and a seam edge's EMF are
//     computed once and enter every cell and face that touches them.
//   - Momentum and B are Cartesian vectors: dU/dt = -(1/V) sum_f s_f F_f |S_f|
//     + S with the faces' area vectors S_f, no geometric source terms.
//   - van Leer PLM (Sect. 2.5) along mesh lines: a face's stencil is its two
//     cells and the cells across their opposite faces, mirrored at a wall;
//     LHLLD / HLLD / HLL (Sect. 2.6) in the face's normal frame, deviation
//     form (Sect. 2.8).
//   - The field lives as face fluxes Phi_f; dPhi_f/dt is minus the
//     circulation of the edge EMFs about the face (Eq. induction).  Edge EMFs
//     are Contact-CT (Sect. 2.4) on E . l over the edge's four faces and
//     cells, upwinded by the faces' mass fluxes; a radial edge at a cube
//     corner (three faces) takes their mean; an edge on a wall has none.
//   - Cell-centred B = (1/V) sum_f s_f Phi_f x_f (divergence theorem on B x).
// Geometry from the factorisation: an angular face of side s between radii
// r0 < r1 has the normal n_s (of the side's great-circle plane) and the area
// (r1^2 - r0^2) theta_s / 2; a radial face of angular cell a at radius r has
// the area r^2 |A_a| along A_a, the vector area of the unit spherical quad;
// cell volumes are (r1^3 - r0^3) Omega_a / 3.
//
// Internal layout: cells c = k NC + a (NC = 6 N^2 angular cells, a = (p N + j)
// N + i); angular faces f = k NS + s (NS = 12 N^2 sides), then radial faces
// FA + k NC + a; radial edges e = k NV + v (NV = 6 N^2 + 2 vertices), then
// angular edges ER + k NS + s.  One thread per cell, face or edge.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <stdexcept>
#include <utility>
#include <vector>

#include "eos_stellar.cuh"
#include "mlp_dev.cuh"
#include "phl.h"
#include "phl_internal.cuh"
#include "riemann.cuh"
#include "riemann_x2.cuh"

using namespace phl;

namespace {

constexpr double PI_S = 3.14159265358979323846;
constexpr int SPT = 256;

// patch frames: centre c, alpha axis a, beta axis b, a x b = c
const int PCI[6][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
const int PAI[6][3] = {{0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 1, 0}};
const int PBI[6][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {-1, 0, 0}, {1, 0, 0}};

struct V3 {
  double x, y, z;
};
__host__ __device__ inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
__host__ __device__ inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline V3 operator*(V3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ inline double dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline V3 cross3(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double len3(V3 a) { return sqrt(dot3(a, a)); }
__host__ __device__ inline V3 unit3(V3 a) { return a * (1.0 / len3(a)); }
__host__ __device__ inline V3 ld3(const double *p, long i) { return v3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }

// ---------------------------------------------------------------------------
// host: the angular mesh

struct Ang {
  int N = 0;
  long NC = 0, NS = 0, NV = 0;
  std::vector<double> vd;              // 3 per vertex: unit direction
  // sides
  std::vector<int> sv0, sv1;           // vertices (sv0 < sv1)
  std::vector<int> sL, sR, sLL, sRR;   // cells on the -n / +n side, and across their opposite sides
  std::vector<double> sn, sl, smid, sth;   // unit normal, chord direction (v0 -> v1), midpoint direction, angle
  std::vector<signed char> s_in, s_v0, s_v1, s_swap;   // boundary orientations; Contact-CT ordering
  // cells
  std::vector<int> cs;                 // 4 per cell: sides -a, +a, -b, +b
  std::vector<signed char> csg, crs;   // 4 per cell: +1 when n_s leaves the cell; orientation in the radial face
  std::vector<double> com, cdc, cna, cva;   // solid angle, centre direction, unit vector area, |vector area|
  // vertices: Contact-CT of the radial edges
  std::vector<unsigned char> vcnt;     // 3 (cube corner) or 4
  std::vector<int> vcell, vside;       // 4 per vertex, cyclic for 4
  std::vector<signed char> vsgn;       // 4 per vertex: +1 when the side's -n cell is the from-cell
  // ABI copies of the angular faces: alpha [p][j][i] (i = 0..N), then beta [p][j][i] (j = 0..N)
  std::vector<int> abi_s;
  std::vector<signed char> abi_sg, abi_own;
};

std::array<int, 3> vcode(int p, int i, int j, int N) {   // grid-line codes in [-N, N] per axis
  std::array<int, 3> c;
  for (int d = 0; d < 3; ++d) c[d] = PCI[p][d] * N + PAI[p][d] * (2 * i - N) + PBI[p][d] * (2 * j - N);
  return c;
}

// the cube-surface point of the codes (tan of q pi / 4N per axis, exactly
// +-1 on the centre axis), normalised
V3 vdir(const std::array<int, 3> &c, int N) {
  double x[3];
  for (int d = 0; d < 3; ++d) {
    const int q = c[d], a = std::abs(q);
    const double t = a == N ? 1.0 : (a == 0 ? 0.0 : tan(a * (PI_S / (4.0 * N))));
    x[d] = q < 0 ? -t : t;
  }
  return unit3(v3(x[0], x[1], x[2]));
}

double tri_solid_angle(V3 a, V3 b, V3 c) {   // Van Oosterom & Strackee (1983)
  return 2.0 * atan2(fabs(dot3(a, cross3(b, c))), 1.0 + dot3(a, b) + dot3(b, c) + dot3(c, a));
}

// vector area of a unit spherical quadrilateral with great-circle sides,
// corners counter-clockwise: half the sum of each side's angle times the unit
// normal of its plane
V3 quad_vector_area(const V3 *d) {
  V3 s = v3(0, 0, 0);
  for (int q = 0; q < 4; ++q) {
    const V3 u = d[q], w = d[(q + 1) % 4], c = cross3(u, w);
    s = s + unit3(c) * (0.5 * atan2(len3(c), dot3(u, w)));
  }
  return s;
}

void build_ang(int N, Ang &M) {
  M.N = N;
  const int N1 = N + 1;
  // vertices (only patch-boundary vertices can be shared)
  std::map<std::array<int, 3>, int> vid;
  std::vector<V3> vd;
  std::vector<int> av(6 * N1 * N1);
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N; ++i) {
        const bool bnd = i == 0 || i == N || j == 0 || j == N;
        const auto c = vcode(p, i, j, N);
        auto it = bnd ? vid.find(c) : vid.end();
        int id;
        if (it == vid.end()) {
          id = (int)vd.size();
          if (bnd) vid[c] = id;
          vd.push_back(vdir(c, N));
        } else {
          id = it->second;
        }
        av[(p * N1 + j) * N1 + i] = id;
      }
  M.NV = (long)vd.size();
  if (M.NV != 6L * N * N + 2) throw std::runtime_error("cubed-sphere vertex count");
  auto AV = [&](int p, int i, int j) { return av[(p * N1 + j) * N1 + i]; };
  auto CELL = [&](int p, int i, int j) { return (p * N + j) * N + i; };
  M.NC = 6L * N * N;
  // sides in ABI order: alpha sides (from (i, j) to (i, j+1)), then beta
  // sides (from (i, j) to (i+1, j)); the first copy fixes the orientation
  M.abi_s.assign(2 * 6 * N * N1, -1);
  M.abi_sg.assign(2 * 6 * N * N1, 1);
  M.abi_own.assign(2 * 6 * N * N1, 0);
  std::map<std::pair<int, int>, int> sid;
  std::vector<V3> nrm;
  long t = 0;
  for (int kind = 0; kind < 2; ++kind)
    for (int p = 0; p < 6; ++p) {
      const int JJ = kind == 1 ? N1 : N, II = kind == 0 ? N1 : N;
      for (int j = 0; j < JJ; ++j)
        for (int i = 0; i < II; ++i, ++t) {
          const int v0 = AV(p, i, j), v1 = kind == 0 ? AV(p, i, j + 1) : AV(p, i + 1, j);
          const int lo = kind == 0 ? (i > 0 ? CELL(p, i - 1, j) : -1) : (j > 0 ? CELL(p, i, j - 1) : -1);
          const int hi = kind == 0 ? (i < N ? CELL(p, i, j) : -1) : (j < N ? CELL(p, i, j) : -1);
          const bool bnd = kind == 0 ? (i == 0 || i == N) : (j == 0 || j == N);
          const int *ax = kind == 0 ? PAI[p] : PBI[p];
          const V3 axv = v3(ax[0], ax[1], ax[2]);
          const std::pair<int, int> key(std::min(v0, v1), std::max(v0, v1));
          auto it = bnd ? sid.find(key) : sid.end();
          if (it != sid.end()) {   // the second copy of a seam side
            const int s = it->second;
            const bool same = dot3(nrm[s], axv) > 0.0;
            M.abi_s[t] = s;
            M.abi_sg[t] = same ? 1 : -1;
            if (lo >= 0) { if (same) M.sL[s] = lo; else M.sR[s] = lo; }
            if (hi >= 0) { if (same) M.sR[s] = hi; else M.sL[s] = hi; }
            continue;
          }
          const int s = (int)M.sv0.size();
          if (bnd) sid[key] = s;
          M.abi_s[t] = s;
          M.abi_own[t] = 1;
          M.sv0.push_back(key.first);
          M.sv1.push_back(key.second);
          V3 n = unit3(cross3(vd[v0], vd[v1]));
          if (dot3(n, axv) < 0.0) n = n * -1.0;
          nrm.push_back(n);
          M.sL.push_back(lo);
          M.sR.push_back(hi);
        }
    }
  M.NS = (long)M.sv0.size();
  if (M.NS != 12L * N * N) throw std::runtime_error("cubed-sphere side count");
  // cells
  M.cs.resize(4 * M.NC);
  M.csg.resize(4 * M.NC);
  M.crs.resize(4 * M.NC);
  M.com.resize(M.NC);
  M.cdc.resize(3 * M.NC);
  M.cna.resize(3 * M.NC);
  M.cva.resize(M.NC);
  const long na = 6L * N * N1;
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const int a = CELL(p, i, j);
        const long u4[4] = {(long)(p * N + j) * N1 + i, (long)(p * N + j) * N1 + i + 1, na + (long)(p * N1 + j) * N + i,
                            na + (long)(p * N1 + j + 1) * N + i};
        for (int m = 0; m < 4; ++m) {
          const int s = M.abi_s[u4[m]];
          M.cs[4 * a + m] = s;
          M.csg[4 * a + m] = M.sL[s] == a ? 1 : -1;
        }
        const V3 d[4] = {vd[AV(p, i, j)], vd[AV(p, i + 1, j)], vd[AV(p, i + 1, j + 1)], vd[AV(p, i, j + 1)]};
        M.com[a] = tri_solid_angle(d[0], d[1], d[2]) + tri_solid_angle(d[0], d[2], d[3]);
        const V3 dc = unit3(d[0] + d[1] + d[2] + d[3]), A = quad_vector_area(d);
        const double Al = len3(A);
        M.cdc[3 * a] = dc.x; M.cdc[3 * a + 1] = dc.y; M.cdc[3 * a + 2] = dc.z;
        M.cna[3 * a] = A.x / Al; M.cna[3 * a + 1] = A.y / Al; M.cna[3 * a + 2] = A.z / Al;
        M.cva[a] = Al;
      }
  // side geometry and stencils
  M.sn.resize(3 * M.NS); M.sl.resize(3 * M.NS); M.smid.resize(3 * M.NS); M.sth.resize(M.NS);
  M.sLL.resize(M.NS); M.sRR.resize(M.NS);
  M.s_in.resize(M.NS); M.s_v0.resize(M.NS); M.s_v1.resize(M.NS); M.s_swap.resize(M.NS);
  auto across_opposite = [&](int a, int s) {   // the cell across a's side opposite to s
    int m = 0;
    for (int q = 0; q < 4; ++q)
      if (M.cs[4 * a + q] == s) m = q;
    const int g = M.cs[4 * a + (m ^ 1)];
    return M.sL[g] == a ? M.sR[g] : M.sL[g];
  };
  for (long s = 0; s < M.NS; ++s) {
    if (M.sL[s] < 0 || M.sR[s] < 0) throw std::runtime_error("cubed-sphere side without two cells");
    const V3 d0 = vd[M.sv0[s]], d1 = vd[M.sv1[s]], n = nrm[s];
    const V3 l = unit3(d1 - d0), mid = unit3(d0 + d1);
    M.sn[3 * s] = n.x; M.sn[3 * s + 1] = n.y; M.sn[3 * s + 2] = n.z;
    M.sl[3 * s] = l.x; M.sl[3 * s + 1] = l.y; M.sl[3 * s + 2] = l.z;
    M.smid[3 * s] = mid.x; M.smid[3 * s + 1] = mid.y; M.smid[3 * s + 2] = mid.z;
    M.sth[s] = atan2(len3(cross3(d0, d1)), dot3(d0, d1));
    M.sLL[s] = across_opposite(M.sL[s], (int)s);
    M.sRR[s] = across_opposite(M.sR[s], (int)s);
    if (M.sLL[s] < 0 || M.sRR[s] < 0) throw std::runtime_error("cubed-sphere stencil");
    // counter-clockwise about n: the edge at the face's inner radius (x_e -
    // x_f along -mid), and the radial edges at v0 and v1 (along d_v - mid)
    M.s_in[s] = dot3(l, cross3(n, mid * -1.0)) > 0.0 ? 1 : -1;
    M.s_v0[s] = dot3(d0, cross3(n, d0 - mid)) > 0.0 ? 1 : -1;
    M.s_v1[s] = dot3(d1, cross3(n, d1 - mid)) > 0.0 ? 1 : -1;
    // Contact-CT about the angular edge (s, k): from c00 = (L, k-1) the
    // a-neighbour is (R, k-1) and the b-neighbour (L, k), unless l . (da x db) < 0
    const V3 dL = ld3(M.cdc.data(), M.sL[s]), dR = ld3(M.cdc.data(), M.sR[s]);
    M.s_swap[s] = dot3(l, cross3(dR - dL, dL)) < 0.0 ? 1 : 0;
  }
  // radial faces: orientation of each side's angular edge about A_a
  for (long a = 0; a < M.NC; ++a) {
    const V3 na_ = ld3(M.cna.data(), a), dc = ld3(M.cdc.data(), a);
    for (int m = 0; m < 4; ++m) {
      const int s = M.cs[4 * a + m];
      M.crs[4 * a + m] = dot3(ld3(M.sl.data(), s), cross3(na_, ld3(M.smid.data(), s) - dc)) > 0.0 ? 1 : -1;
    }
  }
  // vertices: the sides and cells about each radial edge, cyclic
  M.vcnt.assign(M.NV, 0);
  M.vcell.assign(4 * M.NV, -1);
  M.vside.assign(4 * M.NV, -1);
  M.vsgn.assign(4 * M.NV, 0);
  std::vector<int> vs(4 * M.NV, -1);
  for (long s = 0; s < M.NS; ++s)
    for (int v : {M.sv0[s], M.sv1[s]}) {
      if (M.vcnt[v] >= 4) throw std::runtime_error("cubed-sphere vertex with more than four sides");
      vs[4 * v + M.vcnt[v]++] = (int)s;
    }
  for (long v = 0; v < M.NV; ++v) {
    const int n = M.vcnt[v], *S = &vs[4 * v];
    if (n == 3) {
      for (int m = 0; m < 3; ++m) M.vside[4 * v + m] = S[m];
      continue;
    }
    if (n != 4) throw std::runtime_error("cubed-sphere vertex without four sides");
    int cells[8], nc4 = 0;
    for (int m = 0; m < 4; ++m)
      for (int c : {M.sL[S[m]], M.sR[S[m]]}) {
        bool seen = false;
        for (int q = 0; q < nc4; ++q) seen |= cells[q] == c;
        if (!seen) cells[nc4++] = c;
      }
    if (nc4 != 4) throw std::runtime_error("cubed-sphere vertex without four cells");
    auto between = [&](int a, int b) {
      for (int m = 0; m < 4; ++m)
        if ((M.sL[S[m]] == a && M.sR[S[m]] == b) || (M.sL[S[m]] == b && M.sR[S[m]] == a)) return S[m];
      return -1;
    };
    const int c00 = cells[0];
    int X = -1, Y = -1, c11 = -1;
    for (int q = 1; q < 4; ++q)
      if (between(c00, cells[q]) >= 0) { if (X < 0) X = cells[q]; else Y = cells[q]; }
    for (int q = 1; q < 4; ++q)
      if (cells[q] != X && cells[q] != Y) c11 = cells[q];
    if (X < 0 || Y < 0 || c11 < 0) throw std::runtime_error("cubed-sphere vertex cells not cyclic");
    const V3 x00 = ld3(M.cdc.data(), c00);
    const V3 da = ld3(M.cdc.data(), X) - x00, db = ld3(M.cdc.data(), Y) - x00;
    int c10 = X, c01 = Y;
    if (dot3(vd[v], cross3(da, db)) < 0.0) std::swap(c10, c01);
    const int cc[4] = {c00, c10, c11, c01};
    const int ff[4] = {between(c00, c10), between(c10, c11), between(c01, c11), between(c00, c01)};
    const int from[4] = {c00, c10, c01, c00};   // the mass flux counts positive leaving this cell
    for (int m = 0; m < 4; ++m) {
      if (ff[m] < 0) throw std::runtime_error("cubed-sphere vertex faces not cyclic");
      M.vcell[4 * v + m] = cc[m];
      M.vside[4 * v + m] = ff[m];
      M.vsgn[4 * v + m] = M.sL[ff[m]] == from[m] ? 1 : -1;
    }
  }
  M.vd.resize(3 * M.NV);
  for (long v = 0; v < M.NV; ++v) { M.vd[3 * v] = vd[v].x; M.vd[3 * v + 1] = vd[v].y; M.vd[3 * v + 2] = vd[v].z; }
}

// ---------------------------------------------------------------------------
// device
//
// Two forms of the stage.  FP64: every work array in double.  Mixed (the
// paper's mixed-precision form, Sect. 2.8): U^n stays FP64 and a stage
// carries the cells' increments dU = U^(s) - U^n in FP32 (SSP-RK3 has
// a + b = 1 in every stage, so dU^(s) = b (dU^(s-1) - dt R)); primitives are
// formed as FP32 deviations from the background out of an FP64 difference
// U^n - U_hat plus the FP32 increment; fluxes, EMFs and residuals are FP32 on
// FP32 copies of the geometry; the last stage adds the increment to U^n in
// FP64.  The face fluxes keep FP64 stage values, advanced by circulations
// summed in FP64 from the edge EMFs: every edge's term enters its faces as
// the same FP64 product, so the divergence of each cell stays at FP64
// rounding (Eq. divb), as in the FP64 form; an FP32 copy of the stage's face
// fluxes feeds the FP32 kernels.  GB300 runs FP64 at 1/64 of its FP32 rate,
// so the mixed kernels keep FP64 instructions to the few that the form needs.

// deviations per cell: drho, u (3), B (3), dP; the stellar EOS adds
// dgamma_e, dgamma_c (SW_NS)
enum { SW_RHO = 0, SW_U = 1, SW_B = 4, SW_P = 7, SW_N = 8, SW_GE = 8, SW_GC = 9, SW_NS = 10 };

struct SphDev {
  int N, Nr;
  long NC, NS, NV, FA, NF, ER, NE, ncell;
  double gamma, cfl, mach;
  int riemann;
  const double *r;   // Nr + 1 radii
  const double *vd, *sn, *sl, *smid, *sth, *cdc, *cna, *cva, *com;
  const int *sL, *sR, *sLL, *sRR, *sv0, *sv1, *cs, *vcell, *vside;
  const signed char *s_in, *s_v0, *s_v1, *s_swap, *csg, *crs, *vsgn;
  const unsigned char *vcnt;
  const double *rho_c, *p_c, *rho_f, *p_f, *g_c, *heat;   // null when absent
  const double *eh_c;          // P_hat / (gamma - 1) per shell (null without a background)
  FastDiv dNC, dNS, dNV;       // divisions of flat indices (all below 2^31) by NC, NS, NV
  // FP32 copies for the mixed form: geometry, per-radius factors, background
  const float *vd_f, *sn_f, *sl_f, *smid_f, *sth_f, *cdc_f, *cna_f, *cva_f;
  const float *iom_f;          // 1 / Omega per angular cell
  const float *cw_f, *ce_f;    // per angular cell: unit-radius widths (a, b) and their unit directions
  const float *r_f, *rm_f, *hdr2_f, *ish_f, *dr_f;   // r_k, shell middle, (r1^2 - r0^2) / 2, 3 / (r1^3 - r0^3), r1 - r0
  const float *rho_cf, *p_cf, *rho_ff, *p_ff, *g_cf, *heat_f;
  float gf, igm1f, ggm1f, gm1f, machf;
  int *dflag;
  // stellar EOS (Sect. 2.2) with a uniform composition: the table, Abar and
  // Y_e, code density / pressure / specific energy -> g/cm^3, erg/cm^3, erg/g
  int stellar;
  eos::Table tab;
  double abar, ye, rho_u, p_u, e_u, ntol;
  double irho_u, iabar;        // 1 / rho_u, 1 / Abar
  int nmaxit;
  const double *ge_c, *gc_c, *ge_f, *gc_f;   // background gamma_e, gamma_c: shells (Nr), radii (Nr + 1)
  const float *ge_cf, *gc_cf, *ge_ff, *gc_ff;
  const double *T_c;           // the background's temperature per shell (cold-start guess)
  double *T;                   // cell temperatures (internal order); <= 0: none yet
  double *pred;                // mixed form: 8 per cell, each cell's last inversion (eos::Pred, SoA)
  int wq;                      // mixed W: float4 records per cell (2; 3 with the stellar EOS)
  mlp::Dev mlp;                // temperature-guess network (cold starts), when use_mlp
  int use_mlp;
  float mlp_x0;                // its composition input X_0 / (X_0 + X_1)
};

// work arrays of one form (R = double: FP64, float: mixed)
template <typename R>
struct SphWork {
  R *W;             // 8 (10 stellar) deviations per cell: FP64 SoA; mixed two
                    // float4 per cell ((drho, u), (B, dP)), one 16-byte load
                    // each, and (dgamma_e, dgamma_c, 0, 0) for the stellar EOS
  R *FC, *EF;       // 5 integrated fluxes per face, SoA; face EMF: FP64 3 SoA
                    // components, mixed one float4 per face (E, contact sign)
  double *EE;       // edge EMF line integrals L (E . l), FP64 in both forms
  signed char *UP;  // contact direction per face
};

__device__ __forceinline__ double bg_rho(const SphDev &D, int k) { return D.rho_c ? D.rho_c[k] : 0.0; }
__device__ __forceinline__ double bg_p(const SphDev &D, int k) { return D.p_c ? D.p_c[k] : 0.0; }

// The six faces of cell (a, k) in the order -a, +a, -b, +b, -r, +r: index,
// outward sign, centre.
struct CellFaces {
  long f[6];
  double s[6];
  V3 x[6];
};
__device__ __forceinline__ void cell_faces(const SphDev &D, long a, int k, CellFaces &F) {
  const double rm = 0.5 * (D.r[k] + D.r[k + 1]);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int s = D.cs[4 * a + m];
    F.f[m] = (long)k * D.NS + s;
    F.s[m] = D.csg[4 * a + m];
    F.x[m] = ld3(D.smid, s) * rm;
  }
  const V3 dc = ld3(D.cdc, a);
  F.f[4] = D.FA + (long)k * D.NC + a;
  F.s[4] = -1.0;
  F.x[4] = dc * D.r[k];
  F.f[5] = D.FA + (long)(k + 1) * D.NC + a;
  F.s[5] = 1.0;
  F.x[5] = dc * D.r[k + 1];
}

__device__ __forceinline__ double cell_vol(const SphDev &D, long a, int k) {
  const double r0 = D.r[k], r1 = D.r[k + 1];
  return (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 * D.com[a];
}

__global__ void k_sph_prims(SphDev D, SphWork<double> Wk, const double *__restrict__ U, const double *__restrict__ phi) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= D.ncell) return;
  const int k = (int)fastdiv((unsigned)c, D.dNC);
  const long a = c - (long)k * D.NC;
  CellFaces F;
  cell_faces(D, a, k, F);
  V3 B = v3(0, 0, 0);
#pragma unroll
  for (int m = 0; m < 6; ++m) B = B + F.x[m] * (F.s[m] * phi[F.f[m]]);
  B = B * (1.0 / cell_vol(D, a, k));
  const long n = D.ncell;
  const double rho = U[c];
  const V3 u = v3(U[n + c] / rho, U[2 * n + c] / rho, U[3 * n + c] / rho);
  const double P = (D.gamma - 1.0) * (U[4 * n + c] - 0.5 * rho * dot3(u, u) - 0.5 * dot3(B, B));
  if (!(rho > 0.0) || !(P > 0.0)) atomicOr(D.dflag, FLAG_NEG);
  if (!isfinite(rho) || !isfinite(P)) atomicOr(D.dflag, FLAG_NAN);
  Wk.W[SW_RHO * n + c] = rho - bg_rho(D, k);
  Wk.W[(SW_U + 0) * n + c] = u.x; Wk.W[(SW_U + 1) * n + c] = u.y; Wk.W[(SW_U + 2) * n + c] = u.z;
  Wk.W[(SW_B + 0) * n + c] = B.x; Wk.W[(SW_B + 1) * n + c] = B.y; Wk.W[(SW_B + 2) * n + c] = B.z;
  Wk.W[SW_P * n + c] = P - bg_p(D, k);
}

// the CFL rate (Eq. cfl) sum_d (|u . e_d| + c_f(e_d)) / width_d of one cell,
// FP32 on the mixed form's tables
__device__ __forceinline__ float cfl_rate_mx(const SphDev &D, long a, int k, float rho, float P, float ux, float uy,
                                             float uz, float bx, float by, float bz, float gam) {
  const float a2 = gam * P / rho, b2 = (bx * bx + by * by + bz * bz) / rho;
  const float rm = D.rm_f[k];
  float sum = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float ex, ey, ez, w;
    if (d < 2) {
      ex = D.ce_f[6 * a + 3 * d]; ey = D.ce_f[6 * a + 3 * d + 1]; ez = D.ce_f[6 * a + 3 * d + 2];
      w = rm * D.cw_f[2 * a + d];
    } else {
      ex = D.cdc_f[3 * a]; ey = D.cdc_f[3 * a + 1]; ez = D.cdc_f[3 * a + 2];
      w = D.dr_f[k];
    }
    const float bd = bx * ex + by * ey + bz * ez;
    float disc = (a2 + b2) * (a2 + b2) - 4.f * a2 * bd * bd / rho;
    disc = fmaxf(disc, 0.f);
    sum += (fabsf(ux * ex + uy * ey + uz * ez) + sqrtf(0.5f * (a2 + b2 + sqrtf(disc)))) / w;
  }
  return sum;
}

// Mixed form: primitives of U^n + dU (dU null at the first stage) and the
// stage's face fluxes (FP32 copy).  The density and energy deviations start
// from the FP64 differences rho^n - rho_hat and E^n - P_hat / (gamma - 1);
// the rest is FP32.  With dmax, the CFL rate of every cell is folded into
// dmax (the bits of a non-negative double).
__global__ void __launch_bounds__(SPT) k_sph_prims_mx(SphDev D, SphWork<float> Wk, const double *__restrict__ U,
                                                      const float *__restrict__ dU, const float *__restrict__ phif,
                                                      unsigned long long *dmax) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float rate = 0.f;
  if (c < D.ncell) {
    const int k = (int)fastdiv((unsigned)c, D.dNC);
    const long a = c - (long)k * D.NC, n = D.ncell;
    const float rm = D.rm_f[k];
    float bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int s = D.cs[4 * a + m];
      const float w = (D.csg[4 * a + m] > 0 ? rm : -rm) * phif[(long)k * D.NS + s];
      bx += D.smid_f[3 * s] * w; by += D.smid_f[3 * s + 1] * w; bz += D.smid_f[3 * s + 2] * w;
    }
    const float wr = D.r_f[k + 1] * phif[D.FA + (long)(k + 1) * D.NC + a] - D.r_f[k] * phif[D.FA + (long)k * D.NC + a];
    bx += D.cdc_f[3 * a] * wr; by += D.cdc_f[3 * a + 1] * wr; bz += D.cdc_f[3 * a + 2] * wr;
    const float iv = D.iom_f[a] * D.ish_f[k];
    bx *= iv; by *= iv; bz *= iv;
    // FP64 -> FP32 on the integer pipe (d2f_scaled): GB300 converts at the FP64 rate
    float drho = d2f_scaled(D.rho_c ? U[c] - D.rho_c[k] : U[c], 0);
    float dE = d2f_scaled(D.eh_c ? U[4 * n + c] - D.eh_c[k] : U[4 * n + c], 0);
    float mx = d2f_scaled(U[n + c], 0), my = d2f_scaled(U[2 * n + c], 0), mz = d2f_scaled(U[3 * n + c], 0);
    if (dU) {
      drho += dU[c]; dE += dU[4 * n + c];
      mx += dU[n + c]; my += dU[2 * n + c]; mz += dU[3 * n + c];
    }
    const float rhb = D.rho_cf ? D.rho_cf[k] : 0.f, pb = D.p_cf ? D.p_cf[k] : 0.f;
    const float rho = rhb + drho, ir = 1.0f / rho;
    const float ux = mx * ir, uy = my * ir, uz = mz * ir;
    // P - P_hat = (gamma - 1) (E - E_hat - rho u^2 / 2 - B^2 / 2)
    const float dP = D.gm1f * (dE - 0.5f * (mx * ux + my * uy + mz * uz) - 0.5f * (bx * bx + by * by + bz * bz));
    const float P = pb + dP;
    if (!(rho > 0.f) || !(P > 0.f)) atomicOr(D.dflag, FLAG_NEG);
    if (!isfinite(rho) || !isfinite(P)) atomicOr(D.dflag, FLAG_NAN);
    float4 *W4 = reinterpret_cast<float4 *>(Wk.W);
    W4[2 * c] = make_float4(drho, ux, uy, uz);
    W4[2 * c + 1] = make_float4(bx, by, bz, dP);
    if (dmax) {
      rate = cfl_rate_mx(D, a, k, rho, P, ux, uy, uz, bx, by, bz, D.gf);
      if (!(rate == rate)) rate = INFINITY;
    }
  }
  if (dmax) {   // block maximum; non-negative floats order like their bits
    for (int o = 16; o > 0; o >>= 1) rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    __shared__ float red[SPT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
    __syncthreads();
    if (threadIdx.x == 0) {
      float v = 0.f;
      for (int w = 0; w < SPT / 32; ++w) v = fmaxf(v, red[w]);
      atomicMax(dmax, (unsigned long long)__double_as_longlong((double)v));
    }
  }
}

// ---------------------------------------------------------------------------
// stellar EOS on the shell (Sect. 2.2)

// the background's gamma_e, gamma_c at shell k's middle (radial = false) or
// at radius k; gamma without a background
template <typename R>
__device__ __forceinline__ void bg_gammas(const SphDev &D, int k, bool radial, R &ge, R &gc) {
  if constexpr (sizeof(R) == 4) {
    const float *e = radial ? D.ge_ff : D.ge_cf, *g = radial ? D.gc_ff : D.gc_cf;
    ge = e ? e[k] : D.gf;
    gc = g ? g[k] : D.gf;
  } else {
    const double *e = radial ? D.ge_f : D.ge_c, *g = radial ? D.gc_f : D.gc_c;
    ge = e ? e[k] : D.gamma;
    gc = g ? g[k] : D.gamma;
  }
}

// T with P_EoS(rho, T) = P at fixed rho (EOS units): Newton on P from T,
// bracketed in the table's temperature range; o holds the EOS at that T
__device__ bool sph_p_to_T(const eos::Table &t, double rho, double P, double abar, double ye, double &T,
                           eos::EosOut<double> &o) {
  double lo = t.Tlo, hi = t.Thi;
  if (!(T > lo && T < hi)) T = sqrt(lo * hi);
  for (int it = 0; it < 200; ++it) {
    if (!eos::eos_rt<double>(t, rho, T, abar, ye, o)) return false;
    const double dp = P - o.P;
    if (fabs(dp) <= 1e-14 * P) return true;
    if (dp > 0.0) lo = T; else hi = T;
    double Tn = T + dp / o.PT;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    T = Tn;
  }
  return false;
}

// gamma_e, gamma_c and T of the background at the Nr shell middles (i < Nr)
// and the Nr + 1 radii: out[0..] = ge_c, gc_c, T_c (Nr each), ge_f, gc_f
__global__ void k_sph_bg_stellar(SphDev D, const double *rho_c, const double *p_c, const double *rho_f,
                                 const double *p_f, double *out, int *fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, Nr = D.Nr;
  if (i >= 2 * Nr + 1) return;
  const bool radial = i >= Nr;
  const int k = radial ? i - Nr : i;
  const double rho = (radial ? rho_f[k] : rho_c[k]) * D.rho_u, P = (radial ? p_f[k] : p_c[k]) * D.p_u;
  double T = 1e9;
  eos::EosOut<double> o;
  if (!sph_p_to_T(D.tab, rho, P, D.abar, D.ye, T, o)) { atomicOr(fail, 1); return; }
  if (radial) {
    out[3 * Nr + k] = o.ge;
    out[4 * Nr + 1 + k] = o.gc;
  } else {
    out[k] = o.ge;
    out[Nr + k] = o.gc;
    out[2 * Nr + k] = T;
  }
}

// ABI cell u -> internal cell c
__device__ __forceinline__ long sph_cell_of_abi(const SphDev &D, long u) {
  const long per = (long)D.N * D.N;
  const long pk = u / per, rem = u - pk * per;
  const long p = pk / D.Nr, k = pk - p * D.Nr;
  return k * D.NC + p * per + rem;
}

// the method's cell field (1/V) sum_f s_f Phi_f x_f (FP64)
__device__ __forceinline__ V3 cell_field(const SphDev &D, long a, int k, const double *__restrict__ phi) {
  CellFaces F;
  cell_faces(D, a, k, F);
  V3 B = v3(0, 0, 0);
#pragma unroll
  for (int m = 0; m < 6; ++m) B = B + F.x[m] * (F.s[m] * phi[F.f[m]]);
  return B * (1.0 / cell_vol(D, a, k));
}

// primitives (ABI order) -> conserved cells (internal order) and, with the
// stellar EOS, the cells' temperatures
__global__ void k_sph_from_prims(SphDev D, const double *__restrict__ rho_in, const double *__restrict__ vel,
                                 const double *__restrict__ P_in, const double *__restrict__ phi,
                                 double *__restrict__ U) {
  const long u = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (u >= D.ncell) return;
  const long c = sph_cell_of_abi(D, u), n = D.ncell;
  const int k = (int)fastdiv((unsigned)c, D.dNC);
  const long a = c - (long)k * D.NC;
  const V3 B = cell_field(D, a, k, phi);
  const double rho = rho_in[u], P = P_in[u];
  const V3 v = v3(vel[3 * u], vel[3 * u + 1], vel[3 * u + 2]);
  double eden;   // rho e_int
  if (D.stellar) {
    double T = D.T_c ? D.T_c[k] : 1e9;
    eos::EosOut<double> o;
    if (!sph_p_to_T(D.tab, rho * D.rho_u, P * D.p_u, D.abar, D.ye, T, o)) {
      atomicOr(D.dflag, FLAG_NEWTON);
      T = -1.0;
    }
    D.T[c] = T;
    eden = rho * (o.e / D.e_u);
  } else {
    eden = P / (D.gamma - 1.0);
  }
  U[c] = rho;
  U[n + c] = rho * v.x; U[2 * n + c] = rho * v.y; U[3 * n + c] = rho * v.z;
  U[4 * n + c] = eden + 0.5 * rho * dot3(v, v) + 0.5 * dot3(B, B);
}

// ABI <-> internal cell values, nplanes planes of ncell each (temperatures:
// one; the inversion record: eight)
__global__ void k_sph_temps(SphDev D, const double *__restrict__ in, double *__restrict__ out, int to_int,
                            int nplanes = 1) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= nplanes * D.ncell) return;
  const long q = t / D.ncell, u = t - q * D.ncell;
  const long c = q * D.ncell + sph_cell_of_abi(D, u);
  if (to_int) out[c] = in[t];
  else out[t] = in[c];
}

// Cold cells (T <= 0) take the network's guess (cold starts only): warp-
// collective inference on (log10 rho, log10 e_int, X_0) in EOS units from
// U^n and the FP64 face fluxes; the other cells keep their temperature.  No
// thread leaves before the inference (the MMA needs the whole warp).
__global__ void __launch_bounds__(SPT) k_sph_mlp_guess(SphDev D, const double *__restrict__ U,
                                                       const double *__restrict__ phi) {
  const long c0 = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const bool in = c0 < D.ncell;
  const long c = in ? c0 : 0;
  const double T = D.T[c];
  const bool need = in && !(T > 0.0);
  if (!__any_sync(0xffffffffu, need)) return;
  const long n = D.ncell;
  const int k = (int)fastdiv((unsigned)c, D.dNC);
  const long a = c - (long)k * D.NC;
  const V3 B = cell_field(D, a, k, phi);
  const double rho = U[c];
  const V3 m = v3(U[n + c], U[2 * n + c], U[3 * n + c]);
  const double eint = (U[4 * n + c] - 0.5 * dot3(m, m) / rho - 0.5 * dot3(B, B)) / rho;
  const bool ok = rho > 0.0 && eint > 0.0;
  const float lr = ok ? (float)log10(rho * D.rho_u) : D.mlp.c[0];
  const float le = ok ? (float)log10(eint * D.e_u) : D.mlp.c[1];
  const float lt = mlp::guess_log10T(D.mlp, lr, le, D.mlp_x0);
  if (need) D.T[c] = ok ? exp10((double)lt) : (D.T_c ? D.T_c[k] : 1e9);
}

// Stellar primitives: e_int -> T by Newton (Sect. 2.2) from the cell's last
// temperature (the shell background's where it has none), then P, gamma_e,
// gamma_c.  FP64 form (R = double): U is the stage state, the field from the
// FP64 fluxes phi, W in SoA; mixed form (R = float): U^n + dU (FP64 sums: the
// low-Mach deviations need P to ~1e-12), the field from the FP32 fluxes phif,
// FP64 Newton (FP32 iterations first from a far guess, eos_invert_mixed),
// three float4 records per cell, and with dmax the CFL rate folded in.
// pm (mixed form): 1 records each cell's inversion in D.pred, 2 also starts
// from the previous record (eos_invert_rec; the second and third stages).
template <typename R>
__global__ void __launch_bounds__(SPT) k_sph_prims_st(SphDev D, SphWork<R> Wk, const double *__restrict__ U,
                                                      const float *__restrict__ dU, const double *__restrict__ phi,
                                                      const float *__restrict__ phif, unsigned long long *dmax,
                                                      int pm) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float rate = 0.f;
  if (c < D.ncell) {
    const int k = (int)fastdiv((unsigned)c, D.dNC);
    const long a = c - (long)k * D.NC, n = D.ncell;
    double bx, by, bz;
    if constexpr (sizeof(R) == 4) {   // as k_sph_prims_mx
      const float rm = D.rm_f[k];
      float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int s = D.cs[4 * a + m];
        const float w = (D.csg[4 * a + m] > 0 ? rm : -rm) * phif[(long)k * D.NS + s];
        fx += D.smid_f[3 * s] * w; fy += D.smid_f[3 * s + 1] * w; fz += D.smid_f[3 * s + 2] * w;
      }
      const float wr = D.r_f[k + 1] * phif[D.FA + (long)(k + 1) * D.NC + a] - D.r_f[k] * phif[D.FA + (long)k * D.NC + a];
      fx += D.cdc_f[3 * a] * wr; fy += D.cdc_f[3 * a + 1] * wr; fz += D.cdc_f[3 * a + 2] * wr;
      const float iv = D.iom_f[a] * D.ish_f[k];
      // FP32 -> FP64 on the integer pipe (f2d_scaled; GB300 converts at the FP64 rate)
      bx = f2d_scaled(fx * iv, 0); by = f2d_scaled(fy * iv, 0); bz = f2d_scaled(fz * iv, 0);
    } else {
      const V3 B = cell_field(D, a, k, phi);
      bx = B.x; by = B.y; bz = B.z;
    }
    double rho = U[c], mx = U[n + c], my = U[2 * n + c], mz = U[3 * n + c], E = U[4 * n + c];
    if (sizeof(R) == 4 && dU) {
      rho += f2d_scaled(dU[c], 0); mx += f2d_scaled(dU[n + c], 0); my += f2d_scaled(dU[2 * n + c], 0);
      mz += f2d_scaled(dU[3 * n + c], 0); E += f2d_scaled(dU[4 * n + c], 0);
    }
    const double ir = 1.0 / rho;
    const double ux = mx * ir, uy = my * ir, uz = mz * ir;
    const double eint = (E - 0.5 * (mx * ux + my * uy + mz * uz) - 0.5 * (bx * bx + by * by + bz * bz)) * ir;
    double T = D.T[c];
    if (!(T > 0.0)) T = D.T_c ? D.T_c[k] : 1e9;
    eos::EosOut<double> o;
    int it;
    if (sizeof(R) == 4 && pm) {
      eos::Pred pr{};
      double *rp = D.pred + c;
      if (pm == 2) pr = eos::Pred{rp[0], rp[n], rp[2 * n], rp[3 * n], rp[4 * n], rp[5 * n], rp[6 * n], rp[7 * n]};
      it = eos::eos_invert_rec(D.tab, rho * D.rho_u, ir * D.irho_u, eint * D.e_u, D.abar, D.iabar, D.ye, T, D.ntol,
                               D.nmaxit, o, pr, pm == 2);
      rp[0] = pr.rho; rp[n] = pr.e; rp[2 * n] = pr.icv; rp[3 * n] = pr.er;
      rp[4 * n] = pr.lnT; rp[5 * n] = pr.iT; rp[6 * n] = pr.x; rp[7 * n] = pr.ine;
    } else {
      it = sizeof(R) == 8
               ? eos::eos_invert<double>(D.tab, rho * D.rho_u, eint * D.e_u, D.abar, D.ye, T, D.ntol, D.nmaxit, o)
               : eos::eos_invert_mixed(D.tab, rho * D.rho_u, eint * D.e_u, D.abar, D.ye, T, D.ntol, D.nmaxit, o);
    }
    if (it < 0) atomicOr(D.dflag, FLAG_NEWTON);
    D.T[c] = T;
    const double P = o.P / D.p_u;
    if (!(rho > 0.0) || !(P > 0.0)) atomicOr(D.dflag, FLAG_NEG);
    if (!isfinite(rho) || !isfinite(P)) atomicOr(D.dflag, FLAG_NAN);
    double geh, gch;
    bg_gammas<double>(D, k, false, geh, gch);
    const double dP = P - bg_p(D, k), dge = o.ge - geh, dgc = o.gc - gch;
    if constexpr (sizeof(R) == 4) {
      // FP64 -> FP32 on the integer pipe (d2f_scaled)
      float drho = d2f_scaled(D.rho_c ? U[c] - D.rho_c[k] : U[c], 0);
      if (dU) drho += dU[c];
      const float fux = d2f_scaled(ux, 0), fuy = d2f_scaled(uy, 0), fuz = d2f_scaled(uz, 0);
      const float fbx = d2f_scaled(bx, 0), fby = d2f_scaled(by, 0), fbz = d2f_scaled(bz, 0);
      const float fdP = d2f_scaled(dP, 0);
      float4 *W4 = reinterpret_cast<float4 *>(Wk.W);
      W4[3 * c] = make_float4(drho, fux, fuy, fuz);
      W4[3 * c + 1] = make_float4(fbx, fby, fbz, fdP);
      W4[3 * c + 2] = make_float4((float)dge, (float)dgc, 0.f, 0.f);
      if (dmax) {
        const float frho = (D.rho_cf ? D.rho_cf[k] : 0.f) + drho, fP = (D.p_cf ? D.p_cf[k] : 0.f) + fdP;
        rate = cfl_rate_mx(D, a, k, frho, fP, fux, fuy, fuz, fbx, fby, fbz, (float)o.gc);
        if (!(rate == rate)) rate = INFINITY;
      }
    } else {
      Wk.W[SW_RHO * n + c] = rho - bg_rho(D, k);
      Wk.W[(SW_U + 0) * n + c] = ux; Wk.W[(SW_U + 1) * n + c] = uy; Wk.W[(SW_U + 2) * n + c] = uz;
      Wk.W[(SW_B + 0) * n + c] = bx; Wk.W[(SW_B + 1) * n + c] = by; Wk.W[(SW_B + 2) * n + c] = bz;
      Wk.W[SW_P * n + c] = dP;
      Wk.W[SW_GE * n + c] = dge;
      Wk.W[SW_GC * n + c] = dgc;
    }
  }
  if (sizeof(R) == 4 && dmax) {   // block maximum; non-negative floats order like their bits
    for (int o2 = 16; o2 > 0; o2 >>= 1) rate = fmaxf(rate, __shfl_xor_sync(0xffffffffu, rate, o2));
    __shared__ float red[SPT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
    __syncthreads();
    if (threadIdx.x == 0) {
      float v = 0.f;
      for (int w = 0; w < SPT / 32; ++w) v = fmaxf(v, red[w]);
      atomicMax(dmax, (unsigned long long)__double_as_longlong((double)v));
    }
  }
}

// deviations of cell c, mirrored across a wall of unit normal (nx, ny, nz) when mir
template <typename R, bool ST = false>
__device__ __forceinline__ void load_w(const SphDev &D, const SphWork<R> &Wk, long c, bool mir, R nx, R ny, R nz,
                                       R *w) {
  if constexpr (sizeof(R) == 4) {
    const float4 *W4 = reinterpret_cast<const float4 *>(Wk.W) + (ST ? 3 : 2) * c;
    const float4 a = W4[0], b = W4[1];
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    if constexpr (ST) {
      const float4 g = W4[2];
      w[SW_GE] = g.x; w[SW_GC] = g.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < (ST ? SW_NS : SW_N); ++v) w[v] = Wk.W[v * D.ncell + c];
  }
  if (mir) {
    const R un = R(2) * (w[SW_U] * nx + w[SW_U + 1] * ny + w[SW_U + 2] * nz);
    const R bn = R(2) * (w[SW_B] * nx + w[SW_B + 1] * ny + w[SW_B + 2] * nz);
    w[SW_U] -= un * nx; w[SW_U + 1] -= un * ny; w[SW_U + 2] -= un * nz;
    w[SW_B] -= bn * nx; w[SW_B + 1] -= bn * ny; w[SW_B + 2] -= bn * nz;
  }
}

// (FP32: the fast division, the deviations being O(1) in scaled units)
template <typename R>
__device__ __forceinline__ R vl_t(R a, R b, R c) {
  const R dm = b - a, dp = c - b;
  if constexpr (sizeof(R) == 4) return dm * dp > R(0) ? __fdividef(R(2) * dm * dp, dm + dp) : R(0);
  else return dm * dp > R(0) ? R(2) * dm * dp / (dm + dp) : R(0);
}

// Per-face flux of either form.  MX: the mixed form's FP32 tables and face
// fluxes (phif); else FP64 tables and phi.  ST: the stellar EOS (gamma_e,
// gamma_c reconstructed as deviations from the face's background, the
// general-EOS solver).
template <typename R, bool MX, bool ST = false>
__global__ void __launch_bounds__(SPT) k_sph_flux(SphDev D, SphWork<R> Wk, const double *__restrict__ phi,
                                                  const float *__restrict__ phif) {
  const long f = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (f >= D.NF) return;
  constexpr int NW = ST ? SW_NS : SW_N;
  R wL[NW], wR[NW], wLL[NW], wRR[NW];
  R n0, n1, n2, A, brho = R(0), bp = R(0), bge = R(0), bgc = R(0);
  bool wall = false;
  if (f < D.FA) {   // angular face (s, k)
    const int k = (int)fastdiv((unsigned)f, D.dNS);
    const long s = f - (long)k * D.NS, base = (long)k * D.NC;
    load_w<R, ST>(D, Wk, base + D.sL[s], false, R(0), R(0), R(0), wL);
    load_w<R, ST>(D, Wk, base + D.sR[s], false, R(0), R(0), R(0), wR);
    load_w<R, ST>(D, Wk, base + D.sLL[s], false, R(0), R(0), R(0), wLL);
    load_w<R, ST>(D, Wk, base + D.sRR[s], false, R(0), R(0), R(0), wRR);
    if constexpr (ST) bg_gammas<R>(D, k, false, bge, bgc);
    if constexpr (MX) {
      n0 = D.sn_f[3 * s]; n1 = D.sn_f[3 * s + 1]; n2 = D.sn_f[3 * s + 2];
      A = D.hdr2_f[k] * D.sth_f[s];
      if (D.rho_cf) { brho = D.rho_cf[k]; bp = D.p_cf[k]; }
    } else {
      n0 = D.sn[3 * s]; n1 = D.sn[3 * s + 1]; n2 = D.sn[3 * s + 2];
      const double r0 = D.r[k], r1 = D.r[k + 1];
      A = 0.5 * (r1 * r1 - r0 * r0) * D.sth[s];
      if (D.rho_c) { brho = D.rho_c[k]; bp = D.p_c[k]; }
    }
  } else {          // radial face (a, k)
    const long q = f - D.FA;
    const int k = (int)fastdiv((unsigned)q, D.dNC), Nr = D.Nr;
    const long a = q - (long)k * D.NC;
    if constexpr (MX) {
      n0 = D.cna_f[3 * a]; n1 = D.cna_f[3 * a + 1]; n2 = D.cna_f[3 * a + 2];
      A = D.r_f[k] * D.r_f[k] * D.cva_f[a];
      if (D.rho_ff) { brho = D.rho_ff[k]; bp = D.p_ff[k]; }
    } else {
      n0 = D.cna[3 * a]; n1 = D.cna[3 * a + 1]; n2 = D.cna[3 * a + 2];
      A = D.r[k] * D.r[k] * D.cva[a];
      if (D.rho_f) { brho = D.rho_f[k]; bp = D.p_f[k]; }
    }
    const long c0 = a, cst = D.NC;   // cell (a, kk) = c0 + kk cst
    if constexpr (ST) bg_gammas<R>(D, k, true, bge, bgc);
    if (k == 0) {            // inner wall: the ghost side mirrors cells 0 and 1
      wall = true;
      load_w<R, ST>(D, Wk, c0, false, n0, n1, n2, wR);
      load_w<R, ST>(D, Wk, c0 + cst, false, n0, n1, n2, wRR);
      load_w<R, ST>(D, Wk, c0, true, n0, n1, n2, wL);
      load_w<R, ST>(D, Wk, c0 + cst, true, n0, n1, n2, wLL);
    } else if (k == Nr) {    // outer wall
      wall = true;
      load_w<R, ST>(D, Wk, c0 + (Nr - 1) * cst, false, n0, n1, n2, wL);
      load_w<R, ST>(D, Wk, c0 + (Nr - 2) * cst, false, n0, n1, n2, wLL);
      load_w<R, ST>(D, Wk, c0 + (Nr - 1) * cst, true, n0, n1, n2, wR);
      load_w<R, ST>(D, Wk, c0 + (Nr - 2) * cst, true, n0, n1, n2, wRR);
    } else {                 // beside a wall the far cell is the near one's mirror
      load_w<R, ST>(D, Wk, c0 + (k - 1) * cst, false, n0, n1, n2, wL);
      load_w<R, ST>(D, Wk, c0 + k * cst, false, n0, n1, n2, wR);
      if (k >= 2) load_w<R, ST>(D, Wk, c0 + (k - 2) * cst, false, n0, n1, n2, wLL);
      else load_w<R, ST>(D, Wk, c0, true, n0, n1, n2, wLL);
      if (k + 1 <= Nr - 1) load_w<R, ST>(D, Wk, c0 + (k + 1) * cst, false, n0, n1, n2, wRR);
      else load_w<R, ST>(D, Wk, c0 + (Nr - 1) * cst, true, n0, n1, n2, wRR);
    }
  }
  R ql[NW], qr[NW];
#pragma unroll
  for (int v = 0; v < NW; ++v) {
    ql[v] = wL[v] + R(0.5) * vl_t<R>(wLL[v], wL[v], wR[v]);
    qr[v] = wR[v] - R(0.5) * vl_t<R>(wL[v], wR[v], wRR[v]);
  }
  // normal frame: t1 = unit(e_ax x n) for the Cartesian axis least aligned
  // with n, t2 = n x t1
  const R an0 = fabs(n0), an1 = fabs(n1), an2 = fabs(n2);
  const int ax = an1 < an0 ? (an2 < an1 ? 2 : 1) : (an2 < an0 ? 2 : 0);
  R t1x = ax == 0 ? R(0) : (ax == 1 ? n2 : -n1);
  R t1y = ax == 0 ? -n2 : (ax == 1 ? R(0) : n0);
  R t1z = ax == 0 ? n1 : (ax == 1 ? -n0 : R(0));
  const R it = R(1) / sqrt(t1x * t1x + t1y * t1y + t1z * t1z);
  t1x *= it; t1y *= it; t1z *= it;
  const R t2x = n1 * t1z - n2 * t1y, t2y = n2 * t1x - n0 * t1z, t2z = n0 * t1y - n1 * t1x;
  auto dn = [&](const R *q, int o) { return q[o] * n0 + q[o + 1] * n1 + q[o + 2] * n2; };
  auto d1 = [&](const R *q, int o) { return q[o] * t1x + q[o + 1] * t1y + q[o + 2] * t1z; };
  auto d2 = [&](const R *q, int o) { return q[o] * t2x + q[o + 1] * t2y + q[o + 2] * t2z; };
  R wl[RD_X0], wr[RD_X0];
  wl[RD_RHO] = ql[SW_RHO]; wr[RD_RHO] = qr[SW_RHO];
  wl[RD_UN] = dn(ql, SW_U); wl[RD_UT1] = d1(ql, SW_U); wl[RD_UT2] = d2(ql, SW_U);
  wr[RD_UN] = dn(qr, SW_U); wr[RD_UT1] = d1(qr, SW_U); wr[RD_UT2] = d2(qr, SW_U);
  wl[RD_BT1] = d1(ql, SW_B); wl[RD_BT2] = d2(ql, SW_B);
  wr[RD_BT1] = d1(qr, SW_B); wr[RD_BT2] = d2(qr, SW_B);
  wl[RD_P] = ql[SW_P]; wr[RD_P] = qr[SW_P];
  wl[RD_GE] = wl[RD_GC] = wr[RD_GE] = wr[RD_GC] = R(0);
  if (!(brho + wl[RD_RHO] > R(0) && brho + wr[RD_RHO] > R(0) && bp + wl[RD_P] > R(0) && bp + wr[RD_P] > R(0)))
    atomicOr(D.dflag, FLAG_NEG);
  GasK<R> K;
  R mthr, bn;
  if constexpr (MX) {
    K.g = D.gf; K.igm1 = D.igm1f; K.ggm1 = D.ggm1f;
    mthr = D.machf;
    bn = phif[f] / A;
  } else {
    K.g = D.gamma; K.igm1 = 1.0 / (D.gamma - 1.0); K.ggm1 = D.gamma * K.igm1;
    mthr = D.mach;
    bn = phi[f] / A;
  }
  R fl[7];
  int up;
  if constexpr (ST) {   // the general-EOS solver on the reconstructed gamma deviations
    wl[RD_GE] = ql[SW_GE]; wl[RD_GC] = ql[SW_GC];
    wr[RD_GE] = qr[SW_GE]; wr[RD_GC] = qr[SW_GC];
    riemann_dev<R, 0, false>(wl, wr, bn, brho, bp, bge, bgc, 0, D.riemann, mthr, fl, up);
  } else if constexpr (MX) {
    // the mixed form takes the packed-FP32 solver (left and right sides as the
    // two lanes of each f32x2 instruction): same formulas, FP32 rounding apart
    x2::riemann_ideal_lr(wl, wr, bn, brho, bp, D.riemann, mthr, fl, up, K);
  } else {
    riemann_dev<R, 0, true>(wl, wr, bn, brho, bp, K.g, K.g, 0, D.riemann, mthr, fl, up, K);
  }
  if (wall) {   // a symmetry plane: only the normal-momentum flux survives
#pragma unroll
    for (int q = 0; q < 7; ++q)
      if (q != RF_MN) fl[q] = R(0);
    up = 0;
  }
  const long nf = D.NF;
  Wk.FC[f] = A * fl[RF_RHO];
  Wk.FC[nf + f] = A * (n0 * fl[RF_MN] + t1x * fl[RF_MT1] + t2x * fl[RF_MT2]);
  Wk.FC[2 * nf + f] = A * (n1 * fl[RF_MN] + t1y * fl[RF_MT1] + t2y * fl[RF_MT2]);
  Wk.FC[3 * nf + f] = A * (n2 * fl[RF_MN] + t1z * fl[RF_MT1] + t2z * fl[RF_MT2]);
  Wk.FC[4 * nf + f] = A * fl[RF_E];
  // E_f = -n x F_B with F_B = t1 F_bt1 + t2 F_bt2
  const R fbx = t1x * fl[RF_BT1] + t2x * fl[RF_BT2], fby = t1y * fl[RF_BT1] + t2y * fl[RF_BT2],
          fbz = t1z * fl[RF_BT1] + t2z * fl[RF_BT2];
  const R ex = -(n1 * fbz - n2 * fby), ey = -(n2 * fbx - n0 * fbz), ez = -(n0 * fby - n1 * fbx);
  if constexpr (sizeof(R) == 4) {
    reinterpret_cast<float4 *>(Wk.EF)[f] = make_float4(ex, ey, ez, (float)up);
  } else {
    Wk.EF[f] = ex; Wk.EF[nf + f] = ey; Wk.EF[2 * nf + f] = ez;
    Wk.UP[f] = (signed char)up;
  }
}

template <typename R>
__device__ __forceinline__ R efl(const SphDev &D, const SphWork<R> &Wk, long f, R lx, R ly, R lz, int &up) {
  if constexpr (sizeof(R) == 4) {
    const float4 e = reinterpret_cast<const float4 *>(Wk.EF)[f];
    up = (int)e.w;
    return e.x * lx + e.y * ly + e.z * lz;
  } else {
    up = Wk.UP[f];
    return Wk.EF[f] * lx + Wk.EF[D.NF + f] * ly + Wk.EF[2 * D.NF + f] * lz;
  }
}
template <typename R>
__device__ __forceinline__ R ecl(const SphDev &D, const SphWork<R> &Wk, long c, R lx, R ly, R lz) {   // (-u x B) . l
  R ux, uy, uz, bx, by, bz;
  if constexpr (sizeof(R) == 4) {
    const float4 *W4 = reinterpret_cast<const float4 *>(Wk.W) + (long)D.wq * c;
    const float4 a = W4[0], b = W4[1];
    ux = a.y; uy = a.z; uz = a.w; bx = b.x; by = b.y; bz = b.z;
  } else {
    const long n = D.ncell;
    ux = Wk.W[SW_U * n + c]; uy = Wk.W[(SW_U + 1) * n + c]; uz = Wk.W[(SW_U + 2) * n + c];
    bx = Wk.W[SW_B * n + c]; by = Wk.W[(SW_B + 1) * n + c]; bz = Wk.W[(SW_B + 2) * n + c];
  }
  return -((uy * bz - uz * by) * lx + (uz * bx - ux * bz) * ly + (ux * by - uy * bx) * lz);
}

// Contact-CT (Sect. 2.4) on E . l: cells c00, c10, c11, c01 and faces a0
// (c00|c10), b1 (c10|c11), a1 (c01|c11), b0 (c00|c01); ms: mass-flux signs
template <typename R>
__device__ __forceinline__ R contact_ct(const R *Ec, const R *Ef, const int *ms) {
  const R E00 = Ec[0], E10 = Ec[1], E11 = Ec[2], E01 = Ec[3];
  const R Ea0 = Ef[0], Eb1 = Ef[1], Ea1 = Ef[2], Eb0 = Ef[3];
  const int ma0 = ms[0], mb1 = ms[1], ma1 = ms[2], mb0 = ms[3];
  const R h = R(0.5), q = R(0.25);
  const R lo_l = Eb0 - E00, lo_r = Eb1 - E10, up_l = E01 - Eb0, up_r = E11 - Eb1;
  const R dlo = ma0 > 0 ? lo_l : (ma0 < 0 ? lo_r : h * (lo_l + lo_r));
  const R dup = ma1 > 0 ? up_l : (ma1 < 0 ? up_r : h * (up_l + up_r));
  const R le_d = Ea0 - E00, le_u = Ea1 - E01, ri_d = E10 - Ea0, ri_u = E11 - Ea1;
  const R dle = mb0 > 0 ? le_d : (mb0 < 0 ? le_u : h * (le_d + le_u));
  const R dri = mb1 > 0 ? ri_d : (mb1 < 0 ? ri_u : h * (ri_d + ri_u));
  return q * (Ea1 + Ea0 + Eb1 + Eb0) + q * (dlo - dup) + q * (dle - dri);
}

template <typename R, bool MX>
__global__ void __launch_bounds__(SPT) k_sph_emf(SphDev D, SphWork<R> Wk) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= D.NE) return;
  R Ec[4], Ef[4];
  int ms[4];
  double L;   // the edge's length: r1 - r0 (radial), r theta (angular)
  if (e < D.ER) {   // radial edge (v, k)
    const int k = (int)fastdiv((unsigned)e, D.dNV);
    const long v = e - (long)k * D.NV, fb = (long)k * D.NS, cb = (long)k * D.NC;
    L = D.r[k + 1] - D.r[k];
    const R lx = MX ? (R)D.vd_f[3 * v] : (R)D.vd[3 * v];
    const R ly = MX ? (R)D.vd_f[3 * v + 1] : (R)D.vd[3 * v + 1];
    const R lz = MX ? (R)D.vd_f[3 * v + 2] : (R)D.vd[3 * v + 2];
    if (D.vcnt[v] == 3) {   // a cube corner: the mean of the three face EMFs
      R t = R(0);
      int u3;
      for (int m = 0; m < 3; ++m) t += efl<R>(D, Wk, fb + D.vside[4 * v + m], lx, ly, lz, u3);
      Wk.EE[e] = L * (sizeof(R) == 4 ? f2d_scaled((float)(t / R(3)), 0) : (double)(t / R(3)));
      return;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const long f = fb + D.vside[4 * v + m];
      Ec[m] = ecl<R>(D, Wk, cb + D.vcell[4 * v + m], lx, ly, lz);
      int u;
      Ef[m] = efl<R>(D, Wk, f, lx, ly, lz, u);
      ms[m] = D.vsgn[4 * v + m] * u;
    }
  } else {          // angular edge (s, k); none on a wall
    const long q = e - D.ER;
    const int k = (int)fastdiv((unsigned)q, D.dNS);
    const long s = q - (long)k * D.NS;
    if (k == 0 || k == D.Nr) { Wk.EE[e] = 0.0; return; }
    L = D.r[k] * D.sth[s];
    const R lx = MX ? (R)D.sl_f[3 * s] : (R)D.sl[3 * s];
    const R ly = MX ? (R)D.sl_f[3 * s + 1] : (R)D.sl[3 * s + 1];
    const R lz = MX ? (R)D.sl_f[3 * s + 2] : (R)D.sl[3 * s + 2];
    const long cL0 = (long)(k - 1) * D.NC + D.sL[s], cR0 = (long)(k - 1) * D.NC + D.sR[s];
    const long cL1 = (long)k * D.NC + D.sL[s], cR1 = (long)k * D.NC + D.sR[s];
    const long A0 = (long)(k - 1) * D.NS + s, A1 = (long)k * D.NS + s;
    const long RL = D.FA + (long)k * D.NC + D.sL[s], RR = D.FA + (long)k * D.NC + D.sR[s];
    long cc[4], ff[4];
    if (!D.s_swap[s]) {
      cc[0] = cL0; cc[1] = cR0; cc[2] = cR1; cc[3] = cL1;
      ff[0] = A0; ff[1] = RR; ff[2] = A1; ff[3] = RL;
    } else {
      cc[0] = cL0; cc[1] = cL1; cc[2] = cR1; cc[3] = cR0;
      ff[0] = RL; ff[1] = A1; ff[2] = RR; ff[3] = A0;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {   // every face's -n cell is its from-cell here
      Ec[m] = ecl<R>(D, Wk, cc[m], lx, ly, lz);
      Ef[m] = efl<R>(D, Wk, ff[m], lx, ly, lz, ms[m]);
    }
  }
  const R ect = contact_ct<R>(Ec, Ef, ms);
  Wk.EE[e] = L * (sizeof(R) == 4 ? f2d_scaled((float)ect, 0) : (double)ect);
}

// FP64: out = a base + b (in - dt R), R = (1/V) sum_f s_f F_f - S
__global__ void k_sph_update_cells(SphDev D, SphWork<double> Wk, const double *Uin, const double *Ubase, double *Uout,
                                   double a, double b, const double *__restrict__ dtp) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= D.ncell) return;
  const int k = (int)fastdiv((unsigned)c, D.dNC);
  const long an = c - (long)k * D.NC, nc = D.ncell, nf = D.NF;
  CellFaces F;
  cell_faces(D, an, k, F);
  double r[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int m = 0; m < 6; ++m)
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] += F.s[m] * Wk.FC[v * nf + F.f[m]];
  const double iv = 1.0 / cell_vol(D, an, k);
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v] *= iv;
  const double g = D.g_c ? D.g_c[k] : 0.0;
  const V3 gv = ld3(D.cdc, an) * -g;   // radial, inward
  const double drho = Uin[c] - bg_rho(D, k);
  r[1] -= drho * gv.x; r[2] -= drho * gv.y; r[3] -= drho * gv.z;
  double se = Uin[nc + c] * gv.x + Uin[2 * nc + c] * gv.y + Uin[3 * nc + c] * gv.z;
  if (D.heat) se += D.heat[k];
  r[4] -= se;
  const double dt = *dtp;
  double o[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v] = a * Ubase[v * nc + c] + b * (Uin[v * nc + c] - dt * r[v]);
#pragma unroll
  for (int v = 0; v < 5; ++v) Uout[v * nc + c] = o[v];
}

// Mixed: dU_out = b (dU_in - dt R) (dU_in null at the first stage); the last
// stage writes U^n + dU_out into U in FP64
__global__ void __launch_bounds__(SPT) k_sph_update_cells_mx(SphDev D, SphWork<float> Wk, double *U, const float *dUin,
                                                             float *dUout, float b, const double *__restrict__ dtp,
                                                             int last) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= D.ncell) return;
  const int k = (int)fastdiv((unsigned)c, D.dNC);
  const long an = c - (long)k * D.NC, nc = D.ncell, nf = D.NF;
  float du[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) du[v] = dUin ? dUin[v * nc + c] : 0.f;
  long fi[6];
  float sg[6];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    fi[m] = (long)k * D.NS + D.cs[4 * an + m];
    sg[m] = D.csg[4 * an + m];
  }
  fi[4] = D.FA + (long)k * D.NC + an; sg[4] = -1.f;
  fi[5] = D.FA + (long)(k + 1) * D.NC + an; sg[5] = 1.f;
  float r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int m = 0; m < 6; ++m)
#pragma unroll
    for (int v = 0; v < 5; ++v) r[v] += sg[m] * Wk.FC[v * nf + fi[m]];
  const float iv = D.iom_f[an] * D.ish_f[k];
#pragma unroll
  for (int v = 0; v < 5; ++v) r[v] *= iv;
  // sources of the stage input: (rho - rho_hat) g and rho u . g, heating
  const float drho = d2f_scaled(D.rho_c ? U[c] - D.rho_c[k] : U[c], 0) + du[0];
  const float mx = d2f_scaled(U[nc + c], 0) + du[1], my = d2f_scaled(U[2 * nc + c], 0) + du[2],
              mz = d2f_scaled(U[3 * nc + c], 0) + du[3];
  const float g = D.g_cf ? D.g_cf[k] : 0.f;
  const float gx = -g * D.cdc_f[3 * an], gy = -g * D.cdc_f[3 * an + 1], gz = -g * D.cdc_f[3 * an + 2];
  r[1] -= drho * gx; r[2] -= drho * gy; r[3] -= drho * gz;
  float se = mx * gx + my * gy + mz * gz;
  if (D.heat_f) se += D.heat_f[k];
  r[4] -= se;
  const float dt = (float)*dtp;
  float o[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v] = b * (du[v] - dt * r[v]);
  if (last) {
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v * nc + c] += f2d_scaled(o[v], 0);
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) dUout[v * nc + c] = o[v];
  }
}

// the circulation sum_e sigma L (E . l) about face f (Eq. induction), FP64
// in both forms, from the edges' line integrals: every face that has an edge
// adds the same FP64 value with its orientation's sign
// x with the sign of s (s = +1 or -1) flipped in the integer unit: the FP64
// pipe only sees the additions
__device__ __forceinline__ double sgn_mul(signed char s, double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (s < 0 ? (long long)0x8000000000000000ULL : 0LL));
}

__device__ __forceinline__ double circulation(const SphDev &D, const double *__restrict__ EE, long f) {
  if (f < D.FA) {   // angular face (s, k): edges (s, k), (v1, k), (s, k+1), (v0, k)
    const int k = (int)fastdiv((unsigned)f, D.dNS);
    const long s = f - (long)k * D.NS;
    const signed char si = D.s_in[s];
    const double ein = sgn_mul(si, EE[D.ER + (long)k * D.NS + s]);
    const double eout = sgn_mul((signed char)-si, EE[D.ER + (long)(k + 1) * D.NS + s]);
    const double e1 = sgn_mul(D.s_v1[s], EE[(long)k * D.NV + D.sv1[s]]);
    const double e0 = sgn_mul(D.s_v0[s], EE[(long)k * D.NV + D.sv0[s]]);
    return ((ein + eout) + e1) + e0;
  }
  const long q = f - D.FA;   // radial face (a, k): the angular edges (s_m, k)
  const int k = (int)fastdiv((unsigned)q, D.dNC);
  const long an = q - (long)k * D.NC, eb = D.ER + (long)k * D.NS;
  double e[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) e[m] = sgn_mul(D.crs[4 * an + m], EE[eb + D.cs[4 * an + m]]);
  return ((e[0] + e[1]) + e[2]) + e[3];
}

// out = a base + b (in - dt circulation) in FP64; phif (mixed form): the FP32
// copy of out for the next stage's FP32 kernels
__global__ void __launch_bounds__(SPT) k_sph_update_faces(SphDev D, const double *__restrict__ EE, const double *pin,
                                                          const double *pbase, double *pout, double a, double b,
                                                          const double *__restrict__ dtp, float *phif) {
  const long f = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (f >= D.NF) return;
  const double t = circulation(D, EE, f);
  // the first stage (a = 0, b = 1) is in - dt circulation: one FMA
  const double o = a == 0.0 && b == 1.0 ? fma(-*dtp, t, pin[f]) : a * pbase[f] + b * (pin[f] - *dtp * t);
  pout[f] = o;
  if (phif) phif[f] = d2f_scaled(o, 0);
}

__global__ void k_sph_dt(SphDev D, SphWork<double> Wk, unsigned long long *dmax) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double m = 0.0;
  if (c < D.ncell) {
    const long n = D.ncell;
    const int k = (int)fastdiv((unsigned)c, D.dNC);
    const long a = c - (long)k * D.NC;
    const double rho = Wk.W[SW_RHO * n + c] + bg_rho(D, k);
    const double P = Wk.W[SW_P * n + c] + bg_p(D, k);
    const V3 u = v3(Wk.W[SW_U * n + c], Wk.W[(SW_U + 1) * n + c], Wk.W[(SW_U + 2) * n + c]);
    const V3 b = v3(Wk.W[SW_B * n + c], Wk.W[(SW_B + 1) * n + c], Wk.W[(SW_B + 2) * n + c]);
    double gam = D.gamma;
    if (D.stellar) {
      double geh;
      bg_gammas<double>(D, k, false, geh, gam);
      gam += Wk.W[SW_GC * n + c];
    }
    const double a2 = gam * P / rho, b2 = dot3(b, b) / rho;
    CellFaces F;
    cell_faces(D, a, k, F);
    double sum = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {   // the cell's three mesh directions
      const V3 span = F.x[2 * d + 1] - F.x[2 * d];
      const double width = len3(span);
      const V3 ed = span * (1.0 / width);
      const double bd = dot3(b, ed);
      double disc = (a2 + b2) * (a2 + b2) - 4.0 * a2 * bd * bd / rho;
      if (disc < 0.0) disc = 0.0;
      sum += (fabs(dot3(u, ed)) + sqrt(0.5 * (a2 + b2 + sqrt(disc)))) / width;
    }
    m = (sum == sum) ? sum : INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[SPT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < SPT / 32; ++w) v = fmax(v, red[w]);
    atomicMax(dmax, (unsigned long long)__double_as_longlong(v));
  }
}

__global__ void k_sph_dt_fin(double cfl, unsigned long long *dmax, double *dt) {
  const double m = __longlong_as_double((long long)*dmax);
  *dt = m > 0.0 ? cfl / m : 0.0;
  *dmax = 0ull;
}

__global__ void k_sph_set(double v, double *p) { *p = v; }

__global__ void k_sph_to_float(long n, const double *__restrict__ in, float *__restrict__ out) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < n) out[t] = (float)in[t];
}
// ABI <-> internal.  Cells: [v][p][k][j][i] <-> [v][k][a].  Faces: alpha
// [p][k][j][i] (N + 1 per row), beta [p][k][j][i] (N + 1 rows), radial
// [p][k][j][i] (Nr + 1 radii).
struct AbiMap {
  const int *s;
  const signed char *sg, *own;
};

__device__ __forceinline__ long abi_face(const SphDev &D, const AbiMap &M, long t, int &sign, bool &own) {
  const long N = D.N, N1 = N + 1, Nr = D.Nr;
  const long na = 6 * Nr * N * N1;
  if (t < 2 * na) {   // alpha or beta copy: (p, k, rest) -> side entry (kind, p, rest)
    const long kind = t >= na ? 1 : 0;
    const long u = t - kind * na;
    const long per = N * N1;
    const long pk = u / per, rem = u - pk * per;
    const long p = pk / Nr, k = pk - p * Nr;
    const long q = kind * 6 * per + p * per + rem;
    sign = M.sg[q];
    own = M.own[q] != 0;
    return k * D.NS + M.s[q];
  }
  const long u = t - 2 * na, per = N * N;
  const long pk = u / per, rem = u - pk * per;
  const long p = pk / (Nr + 1), k = pk - p * (Nr + 1);
  sign = 1;
  own = true;
  return D.FA + k * D.NC + p * per + rem;
}

__global__ void k_sph_gather_faces(SphDev D, AbiMap M, long n, const double *__restrict__ abi,
                                   double *__restrict__ phi) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int sg;
  bool own;
  const long f = abi_face(D, M, t, sg, own);
  if (own) phi[f] = abi[t];
}
__global__ void k_sph_scatter_faces(SphDev D, AbiMap M, long n, const double *__restrict__ phi,
                                    double *__restrict__ abi) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int sg;
  bool own;
  const long f = abi_face(D, M, t, sg, own);
  abi[t] = sg * phi[f];
}
// to_int: ABI [5][p][k][j][i] -> internal [5][k][a]; else the reverse
__global__ void k_sph_cells(SphDev D, const double *__restrict__ in, double *__restrict__ out, int to_int) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 5 * D.ncell) return;
  const long v = t / D.ncell, u = t - v * D.ncell;   // u: ABI cell index
  const long per = (long)D.N * D.N;
  const long pk = u / per, rem = u - pk * per;
  const long p = pk / D.Nr, k = pk - p * D.Nr;
  const long c = k * D.NC + p * per + rem;
  if (to_int) out[v * D.ncell + c] = in[t];
  else out[t] = in[v * D.ncell + c];
}

inline unsigned nblk(long n) { return (unsigned)((n + SPT - 1) / SPT); }

}  // namespace

struct phl_sphere {
  phl_sphere_desc desc;
  SphDev D;
  SphWork<double> W64{};
  SphWork<float> W32{};
  bool mixed = false;
  AbiMap AM;
  Prof prof;
  cudaStream_t s = nullptr;
  std::vector<void *> allocs;
  double *U = nullptr, *U1 = nullptr, *phi = nullptr, *phi1 = nullptr, *dt = nullptr, *abi_buf = nullptr;
  float *dU = nullptr;     // mixed: the cells' stage increments
  float *phif = nullptr;   // mixed: FP32 copy of the stage's face fluxes
  unsigned long long *dmax = nullptr;
  long nabi = 0;
  long steps = 0;
  bool cold = false;       // stellar: cells without a temperature (the network's guess pending)
  // the step as a CUDA graph (phl_sphere_set_graph): captured for one dt mode
  // (device CFL step, or a fixed dt whose value is part of the capture)
  bool use_graph = false;
  cudaGraphExec_t gexec = nullptr;
  bool g_fixed = false;
  double g_dt = 0.0;
};

namespace {

template <typename T>
cudaError_t up_vec(phl_sphere *S, const T **dst, const std::vector<T> &v) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  S->allocs.push_back(p);
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  *dst = (const T *)p;
  return e;
}
template <typename T>
cudaError_t alloc_n(phl_sphere *S, T **dst, long n) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<long>(1, n) * sizeof(T));
  if (e != cudaSuccess) return e;
  S->allocs.push_back(p);
  e = cudaMemset(p, 0, std::max<long>(1, n) * sizeof(T));
  *dst = (T *)p;
  return e;
}
cudaError_t up_arr(phl_sphere *S, const double **dst, const double *src, long n) {
  if (!src) { *dst = nullptr; return cudaSuccess; }
  return up_vec(S, dst, std::vector<double>(src, src + n));
}
cudaError_t up_arr_f(phl_sphere *S, const float **dst, const double *src, long n) {
  if (!src) { *dst = nullptr; return cudaSuccess; }
  std::vector<float> v(n);
  for (long i = 0; i < n; ++i) v[i] = (float)src[i];
  return up_vec(S, dst, v);
}
std::vector<float> to_f(const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); }

template <typename R>
cudaError_t alloc_work(phl_sphere *S, SphWork<R> &Wk) {
  const SphDev &D = S->D;
  cudaError_t e = alloc_n(S, &Wk.W, (sizeof(R) == 4 ? 4 * D.wq : (D.stellar ? SW_NS : SW_N)) * D.ncell);
  if (e == cudaSuccess) e = alloc_n(S, &Wk.FC, 5 * D.NF);
  if (e == cudaSuccess) e = alloc_n(S, &Wk.EF, (sizeof(R) == 4 ? 4 : 3) * D.NF);
  if (e == cudaSuccess) e = alloc_n(S, &Wk.EE, D.NE);
  if (e == cudaSuccess) e = alloc_n(S, &Wk.UP, sizeof(R) == 4 ? 1 : D.NF);
  return e;
}

phl_status sph_flags(phl_sphere *S) {
  int f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, S->D.dflag, sizeof(int), cudaMemcpyDeviceToHost, S->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "sphere: %s", cudaGetErrorString(e));
  if (f & FLAG_NAN) return (phl_status)set_error(PHL_ENAN, "sphere: non-finite value in the state");
  if (f & FLAG_NEG) return (phl_status)set_error(PHL_ENEGATIVE, "sphere: non-positive density or pressure");
  if (f & FLAG_NEWTON) return (phl_status)set_error(PHL_ENEWTON, "sphere: EOS temperature not found");
  return PHL_OK;
}

// a launch between the timing events of its kernel class (when timing is on)
template <typename F>
void timed(phl_sphere *S, int cls, F &&launch) {
  S->prof.begin(cls, S->s);
  launch();
  S->prof.end(S->s);
}

// The primitives of a stage input: U (FP64 form: the stage state; mixed:
// U^n, with the increments dU from the second stage on), its face fluxes
// (phi FP64, phif the mixed form's FP32 copy); dmax (mixed): fold the CFL
// rate.  A stellar shell whose cells lack temperatures first takes the
// network's guesses (U^n and the FP64 fluxes of the state).
// The stellar mixed form starts each inversion from the cell's record
// (k_sph_prims_st pm = 2; a cleared record gives the plain start).
void sph_prims(phl_sphere *S, const double *U, const float *dU, const double *phi, unsigned long long *dmax,
               int pm = 2) {
  const SphDev &D = S->D;
  timed(S, KC_SPH_PRIM, [&] {
    if (S->cold && D.use_mlp) k_sph_mlp_guess<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->U, S->phi);
    S->cold = false;
    if (D.stellar) {
      if (S->mixed)
        k_sph_prims_st<float><<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W32, U, dU, nullptr, S->phif, dmax,
                                                              D.pred ? pm : 0);
      else k_sph_prims_st<double><<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W64, U, nullptr, phi, nullptr, nullptr, 0);
    } else if (S->mixed) {
      k_sph_prims_mx<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W32, U, dU, S->phif, dmax);
    } else {
      k_sph_prims<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W64, U, phi);
    }
  });
}

// the CFL step of U^n (Eq. cfl) into S->dt; leaves the primitives of U^n in W
void sph_dt(phl_sphere *S) {
  const SphDev &D = S->D;
  if (S->mixed) {   // folded into the primitives
    sph_prims(S, S->U, nullptr, S->phi, S->dmax);
    timed(S, KC_SPH_DT, [&] { k_sph_dt_fin<<<1, 1, 0, S->s>>>(D.cfl, S->dmax, S->dt); });
    return;
  }
  sph_prims(S, S->U, nullptr, S->phi, nullptr);
  timed(S, KC_SPH_DT, [&] {
    k_sph_dt<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W64, S->dmax);
    k_sph_dt_fin<<<1, 1, 0, S->s>>>(D.cfl, S->dmax, S->dt);
  });
}

}  // namespace

extern "C" {

phl_status phl_sphere_create(const phl_sphere_desc *d, phl_sphere **out) {
  if (!d || !out) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: null argument");
  *out = nullptr;
  if (d->N < 2 || d->Nr < 2 || !(d->r_in > 0.0) || !(d->r_out > d->r_in) || !(d->gamma > 1.0) || !(d->cfl > 0.0) ||
      !(d->mach_thr > 0.0))
    return (phl_status)set_error(PHL_EINVAL,
                                 "phl_sphere_create: need N, Nr >= 2, 0 < r_in < r_out, gamma > 1, cfl > 0, mach_thr > 0");
  if (d->riemann < PHL_LHLLD || d->riemann > PHL_HLL)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: bad solver");
  if (d->precision != PHL_FP64 && d->precision != PHL_MIXED)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: bad precision");
  if (d->eos != PHL_EOS_IDEAL && d->eos != PHL_EOS_STELLAR)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: bad eos");
  if (d->eos == PHL_EOS_STELLAR) {
    bool ok = d->eos_table && d->nspec >= 1 && d->nspec <= PHL_MAXSPEC && d->rho_unit > 0.0 && d->p_unit > 0.0;
    double xs = 0.0;
    for (int l = 0; ok && l < d->nspec; ++l) {
      ok = d->A[l] > 0.0 && d->Z[l] > 0.0 && d->X[l] >= 0.0;
      xs += d->X[l];
    }
    if (!ok || !(xs > 0.0))
      return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: the stellar EOS needs eos_table, nspec 1..%d, "
                                               "A, Z > 0, X >= 0 (not all 0), rho_unit, p_unit > 0", PHL_MAXSPEC);
  }
  const bool any = d->rho_c || d->p_c || d->rho_f || d->p_f, all = d->rho_c && d->p_c && d->rho_f && d->p_f;
  if (any && !all) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: the background needs all four profiles");
  // face and edge indices must fit int32 per shell and long overall
  const double nf = 12.0 * d->N * d->N * d->Nr + 6.0 * d->N * d->N * (d->Nr + 1.0);
  const double ne = (6.0 * d->N * d->N + 2.0) * d->Nr + 12.0 * d->N * d->N * (d->Nr + 1.0);
  if (nf > 2147483647.0 || ne > 2147483647.0 || d->N > 8192)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: more than 2^31 faces or edges");
  phl_sphere *S = new phl_sphere();
  S->desc = *d;
  S->s = (cudaStream_t)d->stream;
  S->mixed = d->precision == PHL_MIXED;
  Ang M;
  try {
    build_ang(d->N, M);
  } catch (const std::exception &ex) {
    delete S;
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_create: %s", ex.what());
  }
  SphDev &D = S->D;
  const int Nr = d->Nr;
  D.N = d->N; D.Nr = Nr;
  D.NC = M.NC; D.NS = M.NS; D.NV = M.NV;
  D.ncell = M.NC * Nr;
  D.FA = M.NS * Nr;
  D.NF = D.FA + M.NC * (Nr + 1);
  D.ER = M.NV * Nr;
  D.NE = D.ER + M.NS * (Nr + 1);
  D.gamma = d->gamma; D.cfl = d->cfl; D.mach = d->mach_thr; D.riemann = d->riemann;
  D.dNC = make_fastdiv((unsigned)D.NC); D.dNS = make_fastdiv((unsigned)D.NS); D.dNV = make_fastdiv((unsigned)D.NV);
  D.gf = (float)d->gamma; D.gm1f = (float)(d->gamma - 1.0); D.igm1f = (float)(1.0 / (d->gamma - 1.0));
  D.ggm1f = (float)(d->gamma / (d->gamma - 1.0)); D.machf = (float)d->mach_thr;
  std::vector<double> r(Nr + 1);
  for (int k = 0; k <= Nr; ++k) r[k] = d->r_in + (d->r_out - d->r_in) * k / Nr;
  cudaError_t e = up_vec(S, &D.r, r);
  auto U = [&](auto **dst, const auto &v) { if (e == cudaSuccess) e = up_vec(S, dst, v); };
  U(&D.vd, M.vd); U(&D.sn, M.sn); U(&D.sl, M.sl); U(&D.smid, M.smid); U(&D.sth, M.sth);
  U(&D.cdc, M.cdc); U(&D.cna, M.cna); U(&D.cva, M.cva); U(&D.com, M.com);
  U(&D.sL, M.sL); U(&D.sR, M.sR); U(&D.sLL, M.sLL); U(&D.sRR, M.sRR); U(&D.sv0, M.sv0); U(&D.sv1, M.sv1);
  U(&D.cs, M.cs); U(&D.vcell, M.vcell); U(&D.vside, M.vside);
  U(&D.s_in, M.s_in); U(&D.s_v0, M.s_v0); U(&D.s_v1, M.s_v1); U(&D.s_swap, M.s_swap);
  U(&D.csg, M.csg); U(&D.crs, M.crs); U(&D.vsgn, M.vsgn); U(&D.vcnt, M.vcnt);
  U(&S->AM.s, M.abi_s); U(&S->AM.sg, M.abi_sg); U(&S->AM.own, M.abi_own);
  if (e == cudaSuccess) e = up_arr(S, &D.rho_c, d->rho_c, Nr);
  if (e == cudaSuccess) e = up_arr(S, &D.p_c, d->p_c, Nr);
  if (e == cudaSuccess) e = up_arr(S, &D.rho_f, d->rho_f, Nr + 1);
  if (e == cudaSuccess) e = up_arr(S, &D.p_f, d->p_f, Nr + 1);
  if (e == cudaSuccess) e = up_arr(S, &D.g_c, d->g_c, Nr);
  if (e == cudaSuccess) e = up_arr(S, &D.heat, d->heat, Nr);
  D.eh_c = nullptr;
  if (d->p_c) {
    std::vector<double> eh(Nr);
    for (int k = 0; k < Nr; ++k) eh[k] = d->p_c[k] / (d->gamma - 1.0);
    U(&D.eh_c, eh);
  }
  D.wq = 2;
  if (d->eos == PHL_EOS_STELLAR && e == cudaSuccess) {
    D.stellar = 1;
    D.wq = 3;
    D.tab = *eos_table_view(d->eos_table);
    double inv_abar = 0.0, ye = 0.0;
    for (int l = 0; l < d->nspec; ++l) {
      inv_abar += d->X[l] / d->A[l];
      ye += d->X[l] * d->Z[l] / d->A[l];
    }
    D.abar = 1.0 / inv_abar;
    D.iabar = inv_abar;
    D.ye = ye;
    D.rho_u = d->rho_unit; D.p_u = d->p_unit; D.e_u = d->p_unit / d->rho_unit; D.irho_u = 1.0 / d->rho_unit;
    D.ntol = d->newton_tol > 0.0 ? d->newton_tol : 1e-11;
    D.nmaxit = d->newton_maxit > 0 ? d->newton_maxit : 50;
    if (d->mlp) {
      D.use_mlp = 1;
      D.mlp = mlp_view(d->mlp);
      D.mlp_x0 = (float)(d->nspec > 1 ? d->X[0] / (d->X[0] + d->X[1]) : 1.0);
    }
    e = alloc_n(S, &D.T, D.ncell);
    if (e == cudaSuccess && S->mixed) e = alloc_n(S, &D.pred, 8 * D.ncell);
    if (e == cudaSuccess && d->rho_c) {   // the background's gamma_e, gamma_c and T from the EOS
      double *bg = nullptr;
      int *fail = nullptr;
      e = alloc_n(S, &bg, 5L * Nr + 2);
      if (e == cudaSuccess) e = alloc_n(S, &fail, 1);
      if (e == cudaSuccess) {
        k_sph_bg_stellar<<<(2 * Nr + 1 + 63) / 64, 64>>>(D, D.rho_c, D.p_c, D.rho_f, D.p_f, bg, fail);
        e = cudaGetLastError();
      }
      std::vector<double> h(5L * Nr + 2);
      int f = 0;
      if (e == cudaSuccess) e = cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(h.data(), bg, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && f) {
        phl_sphere_destroy(S);
        return (phl_status)set_error(PHL_ENEWTON, "phl_sphere_create: no EOS temperature for the background");
      }
      D.ge_c = bg; D.gc_c = bg + Nr; D.T_c = bg + 2 * Nr; D.ge_f = bg + 3 * Nr; D.gc_f = bg + 4 * Nr + 1;
      if (S->mixed && e == cudaSuccess) {
        U(&D.ge_cf, std::vector<float>(h.begin(), h.begin() + Nr));
        U(&D.gc_cf, std::vector<float>(h.begin() + Nr, h.begin() + 2 * Nr));
        U(&D.ge_ff, std::vector<float>(h.begin() + 3 * Nr, h.begin() + 4 * Nr + 1));
        U(&D.gc_ff, std::vector<float>(h.begin() + 4 * Nr + 1, h.end()));
      }
    }
  }
  if (S->mixed) {   // FP32 copies of the geometry, radial factors and profiles
    std::vector<float> iom(M.NC), cw(2 * M.NC), ce(6 * M.NC);
    for (long a = 0; a < M.NC; ++a) {
      iom[a] = (float)(1.0 / M.com[a]);
      for (int dd = 0; dd < 2; ++dd) {   // the a and b directions: between the centres of opposite sides
        const V3 span = ld3(M.smid.data(), M.cs[4 * a + 2 * dd + 1]) - ld3(M.smid.data(), M.cs[4 * a + 2 * dd]);
        const double w = len3(span);
        cw[2 * a + dd] = (float)w;
        ce[6 * a + 3 * dd] = (float)(span.x / w); ce[6 * a + 3 * dd + 1] = (float)(span.y / w);
        ce[6 * a + 3 * dd + 2] = (float)(span.z / w);
      }
    }
    std::vector<float> rf(Nr + 1), rmf(Nr), hdr2(Nr), ish(Nr), drf(Nr);
    for (int k = 0; k <= Nr; ++k) rf[k] = (float)r[k];
    for (int k = 0; k < Nr; ++k) {
      rmf[k] = (float)(0.5 * (r[k] + r[k + 1]));
      hdr2[k] = (float)(0.5 * (r[k + 1] * r[k + 1] - r[k] * r[k]));
      ish[k] = (float)(3.0 / (r[k + 1] * r[k + 1] * r[k + 1] - r[k] * r[k] * r[k]));
      drf[k] = (float)(r[k + 1] - r[k]);
    }
    U(&D.vd_f, to_f(M.vd)); U(&D.sn_f, to_f(M.sn)); U(&D.sl_f, to_f(M.sl)); U(&D.smid_f, to_f(M.smid));
    U(&D.sth_f, to_f(M.sth)); U(&D.cdc_f, to_f(M.cdc)); U(&D.cna_f, to_f(M.cna)); U(&D.cva_f, to_f(M.cva));
    U(&D.iom_f, iom); U(&D.cw_f, cw); U(&D.ce_f, ce);
    U(&D.r_f, rf); U(&D.rm_f, rmf); U(&D.hdr2_f, hdr2); U(&D.ish_f, ish); U(&D.dr_f, drf);
    if (e == cudaSuccess) e = up_arr_f(S, &D.rho_cf, d->rho_c, Nr);
    if (e == cudaSuccess) e = up_arr_f(S, &D.p_cf, d->p_c, Nr);
    if (e == cudaSuccess) e = up_arr_f(S, &D.rho_ff, d->rho_f, Nr + 1);
    if (e == cudaSuccess) e = up_arr_f(S, &D.p_ff, d->p_f, Nr + 1);
    if (e == cudaSuccess) e = up_arr_f(S, &D.g_cf, d->g_c, Nr);
    if (e == cudaSuccess) e = up_arr_f(S, &D.heat_f, d->heat, Nr);
  }
  if (e == cudaSuccess) e = alloc_n(S, &D.dflag, 1);
  if (e == cudaSuccess) e = S->mixed ? alloc_work(S, S->W32) : alloc_work(S, S->W64);
  if (e == cudaSuccess) e = alloc_n(S, &S->U, 5 * D.ncell);
  if (e == cudaSuccess) e = alloc_n(S, &S->phi, D.NF);
  if (e == cudaSuccess) e = alloc_n(S, &S->phi1, D.NF);
  if (S->mixed) {
    if (e == cudaSuccess) e = alloc_n(S, &S->dU, 5 * D.ncell);
    if (e == cudaSuccess) e = alloc_n(S, &S->phif, D.NF);
  } else {
    if (e == cudaSuccess) e = alloc_n(S, &S->U1, 5 * D.ncell);
  }
  if (e == cudaSuccess) e = alloc_n(S, &S->dt, 1);
  if (e == cudaSuccess) e = alloc_n(S, &S->dmax, 1);
  S->nabi = 2L * 6 * Nr * d->N * (d->N + 1) + 6L * (Nr + 1) * d->N * d->N;
  if (e == cudaSuccess) e = alloc_n(S, &S->abi_buf, std::max<long>(S->nabi, 5 * D.ncell));
  if (e != cudaSuccess) {
    cudaGetLastError();
    phl_sphere_destroy(S);
    return (phl_status)set_error(PHL_ENOMEM, "phl_sphere_create: %s", cudaGetErrorString(e));
  }
  *out = S;
  return PHL_OK;
}

void phl_sphere_destroy(phl_sphere *S) {
  if (!S) return;
  if (S->gexec) cudaGraphExecDestroy(S->gexec);
  S->prof.release();
  for (void *p : S->allocs) cudaFree(p);
  delete S;
}

phl_status phl_sphere_set_timing(phl_sphere *S, int on) {
  if (!S) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_timing: null sphere");
  S->prof.on = on != 0;
  return PHL_OK;
}

phl_status phl_sphere_kernel_times(phl_sphere *S, phl_kernel_time *out, int max, int *n, int reset) {
  if (!S || !n || (max > 0 && !out)) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_kernel_times: null argument");
  cudaError_t e = S->prof.fold();
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_kernel_times: %s", cudaGetErrorString(e));
  int k = 0;
  for (int c = 0; c < KC_COUNT; ++c) {
    if (S->prof.cnt[c] == 0) continue;
    if (k < max) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kclass_name(c), sizeof(out[k].name) - 1);
      out[k].launches = S->prof.cnt[c];
      out[k].ms = S->prof.ms[c];
    }
    ++k;
  }
  *n = k;
  if (reset)
    for (int c = 0; c < KC_COUNT; ++c) { S->prof.cnt[c] = 0; S->prof.ms[c] = 0.0; }
  return PHL_OK;
}

phl_status phl_sphere_counts(const phl_sphere *S, long *cells, long *faces, long *edges) {
  if (!S) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_counts: null sphere");
  if (cells) *cells = S->D.ncell;
  if (faces) *faces = S->D.NF;
  if (edges) *edges = S->D.NE;
  return PHL_OK;
}

phl_status phl_sphere_set_state(phl_sphere *S, const double *cons, const double *pa, const double *pb,
                                const double *pr, int where) {
  if (!S || !cons || !pa || !pb || !pr) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_state: null argument");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_state: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const long N = S->D.N, Nr = S->D.Nr, na = 6 * Nr * N * (N + 1), nr = 6 * (Nr + 1) * N * N;
  const long nc5 = 5 * S->D.ncell;
  cudaError_t e = cudaMemcpyAsync(S->abi_buf, cons, nc5 * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_cells<<<nblk(nc5), SPT, 0, S->s>>>(S->D, S->abi_buf, S->U, 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf, pa, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + na, pb, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + 2 * na, pr, nr * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_gather_faces<<<nblk(S->nabi), SPT, 0, S->s>>>(S->D, S->AM, S->nabi, S->abi_buf, S->phi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && S->mixed) {
    k_sph_to_float<<<nblk(S->D.NF), SPT, 0, S->s>>>(S->D.NF, S->phi, S->phif);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && S->D.stellar) {   // no temperatures yet: a cold start
    e = cudaMemsetAsync(S->D.T, 0, S->D.ncell * sizeof(double), S->s);
    S->cold = true;
  }
  if (e == cudaSuccess && S->D.pred) e = cudaMemsetAsync(S->D.pred, 0, 8 * S->D.ncell * sizeof(double), S->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S->D.dflag, 0, sizeof(int), S->s);
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_set_state: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_set_prims(phl_sphere *S, const double *rho, const double *vel, const double *P,
                                const double *pa, const double *pb, const double *pr, int where) {
  if (!S || !rho || !vel || !P || !pa || !pb || !pr)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_prims: null argument");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_prims: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const SphDev &D = S->D;
  const long N = D.N, Nr = D.Nr, na = 6 * Nr * N * (N + 1), nr = 6 * (Nr + 1) * N * N, nc = D.ncell;
  cudaError_t e = cudaMemcpyAsync(S->abi_buf, pa, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + na, pb, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + 2 * na, pr, nr * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_gather_faces<<<nblk(S->nabi), SPT, 0, S->s>>>(D, S->AM, S->nabi, S->abi_buf, S->phi);
    e = cudaGetLastError();
  }
  // the primitives in the buffer: rho, P, then vel (3 per cell)
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf, rho, nc * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + nc, P, nc * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->abi_buf + 2 * nc, vel, 3 * nc * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(D.dflag, 0, sizeof(int), S->s);
  if (e == cudaSuccess) {
    k_sph_from_prims<<<nblk(nc), SPT, 0, S->s>>>(D, S->abi_buf, S->abi_buf + 2 * nc, S->abi_buf + nc, S->phi, S->U);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && S->mixed) {
    k_sph_to_float<<<nblk(D.NF), SPT, 0, S->s>>>(D.NF, S->phi, S->phif);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && D.pred) e = cudaMemsetAsync(D.pred, 0, 8 * D.ncell * sizeof(double), S->s);
  S->cold = false;
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_set_prims: %s", cudaGetErrorString(e));
  return where == PHL_HOST ? sph_flags(S) : PHL_OK;
}

phl_status phl_sphere_set_temperature(phl_sphere *S, const double *T, int where) {
  if (!S || !T) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_temperature: null argument");
  if (!S->D.stellar) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_temperature: an ideal-gas shell");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_temperature: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(S->abi_buf, T, S->D.ncell * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_temps<<<nblk(S->D.ncell), SPT, 0, S->s>>>(S->D, S->abi_buf, S->D.T, 1);
    e = cudaGetLastError();
  }
  S->cold = true;   // any value <= 0 marks a cell without one
  if (e == cudaSuccess && S->D.pred) e = cudaMemsetAsync(S->D.pred, 0, 8 * S->D.ncell * sizeof(double), S->s);
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_set_temperature: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_get_eos_record(phl_sphere *S, double *rec, int where) {
  if (!S || !rec) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_eos_record: null argument");
  if (!S->D.pred) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_eos_record: no record (mixed stellar shells)");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_eos_record: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const long n = 8 * S->D.ncell;
  double *buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, n * sizeof(double), S->s);
  if (e == cudaSuccess) {
    k_sph_temps<<<nblk(n), SPT, 0, S->s>>>(S->D, S->D.pred, buf, 0, 8);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(rec, buf, n * sizeof(double), kd, S->s);
  if (buf) cudaFreeAsync(buf, S->s);
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_get_eos_record: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_set_eos_record(phl_sphere *S, const double *rec, int where) {
  if (!S || !rec) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_eos_record: null argument");
  if (!S->D.pred) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_eos_record: no record (mixed stellar shells)");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_eos_record: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const long n = 8 * S->D.ncell;
  double *buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, n * sizeof(double), S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, rec, n * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_temps<<<nblk(n), SPT, 0, S->s>>>(S->D, buf, S->D.pred, 1, 8);
    e = cudaGetLastError();
  }
  if (buf) cudaFreeAsync(buf, S->s);
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_set_eos_record: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_get_temperature(phl_sphere *S, double *T, int where) {
  if (!S || !T) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_temperature: null argument");
  if (!S->D.stellar) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_temperature: an ideal-gas shell");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_temperature: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  k_sph_temps<<<nblk(S->D.ncell), SPT, 0, S->s>>>(S->D, S->D.T, S->abi_buf, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(T, S->abi_buf, S->D.ncell * sizeof(double), kd, S->s);
  if (e == cudaSuccess && where == PHL_HOST) e = cudaStreamSynchronize(S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_get_temperature: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_get_state(phl_sphere *S, double *cons, double *pa, double *pb, double *pr, int where) {
  if (!S || !cons || !pa || !pb || !pr) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_state: null argument");
  if (where != PHL_HOST && where != PHL_DEVICE)
    return (phl_status)set_error(PHL_EINVAL, "phl_sphere_get_state: bad where");
  const cudaMemcpyKind kd = where == PHL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const long N = S->D.N, Nr = S->D.Nr, na = 6 * Nr * N * (N + 1), nr = 6 * (Nr + 1) * N * N;
  const long nc5 = 5 * S->D.ncell;
  k_sph_cells<<<nblk(nc5), SPT, 0, S->s>>>(S->D, S->U, S->abi_buf, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(cons, S->abi_buf, nc5 * sizeof(double), kd, S->s);
  if (e == cudaSuccess) {
    k_sph_scatter_faces<<<nblk(S->nabi), SPT, 0, S->s>>>(S->D, S->AM, S->nabi, S->phi, S->abi_buf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(pa, S->abi_buf, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pb, S->abi_buf + na, na * sizeof(double), kd, S->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pr, S->abi_buf + 2 * na, nr * sizeof(double), kd, S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_get_state: %s", cudaGetErrorString(e));
  return sph_flags(S);
}

phl_status phl_sphere_compute_dt(phl_sphere *S, double *dt_out) {
  if (!S || !dt_out) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_compute_dt: null argument");
  sph_dt(S);
  cudaError_t e = cudaMemcpyAsync(dt_out, S->dt, sizeof(double), cudaMemcpyDeviceToHost, S->s);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_compute_dt: %s", cudaGetErrorString(e));
  return sph_flags(S);
}

phl_status phl_sphere_set_graph(phl_sphere *S, int on) {
  if (!S) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_graph: null sphere");
  if (on && !S->s) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_set_graph: needs a stream of its own");
  S->use_graph = on != 0;
  if (!S->use_graph && S->gexec) {
    cudaGraphExecDestroy(S->gexec);
    S->gexec = nullptr;
  }
  return PHL_OK;
}

}  // extern "C"

namespace {
void sph_steps(phl_sphere *S, double dt, int nsteps);

// The step captured as a graph, for the current dt mode; false: not
// available (the caller launches the kernels directly).
bool sph_graph(phl_sphere *S, double dt) {
  const bool fixed = dt > 0.0;
  if (S->gexec && S->g_fixed == fixed && (!fixed || dt == S->g_dt)) return true;
  if (S->gexec) {
    cudaGraphExecDestroy(S->gexec);
    S->gexec = nullptr;
  }
  if (cudaStreamBeginCapture(S->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  sph_steps(S, dt, 1);
  cudaGraph_t g = nullptr;
  const cudaError_t e1 = cudaGetLastError(), e2 = cudaStreamEndCapture(S->s, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  const cudaError_t e3 = cudaGraphInstantiate(&S->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    cudaGetLastError();
    S->gexec = nullptr;
    return false;
  }
  S->g_fixed = fixed;
  S->g_dt = dt;
  return true;
}

// nsteps SSP-RK3 steps by direct launches
void sph_steps(phl_sphere *S, double dt, int nsteps) {
  static const double A3[3] = {0.0, 0.75, 1.0 / 3.0}, B3[3] = {1.0, 0.25, 2.0 / 3.0};
  const SphDev &D = S->D;
  for (int n = 0; n < nsteps; ++n) {
    if (dt > 0.0) timed(S, KC_SCALAR, [&] { k_sph_set<<<1, 1, 0, S->s>>>(dt, S->dt); });
    else sph_dt(S);   // leaves the primitives of U^n for the first stage
    // Shu-Osher SSP-RK3 (Sect. 2.9)
    for (int st = 0; st < 3; ++st) {
      const bool last = st == 2, prims = st > 0 || dt > 0.0;
      // faces (both forms): stage input phi1 (Phi^n at the first stage),
      // out = a Phi^n + b (in - dt circulation); each thread reads its own
      // element of in and base before writing out
      const double *pin = st == 0 ? S->phi : S->phi1;
      double *pout = last ? S->phi : S->phi1;
      const double a = A3[st], b = B3[st];
      if (S->mixed) {
        // cells: stage input U^n + dU; increments out dU = b (dU - dt R)
        const float *dUin = st == 0 ? nullptr : S->dU;
        if (prims) sph_prims(S, S->U, dUin, pin, nullptr);
        timed(S, KC_SPH_FLUX, [&] {
          if (D.stellar) k_sph_flux<float, true, true><<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W32, pin, S->phif);
          else k_sph_flux<float, true><<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W32, pin, S->phif);
        });
        timed(S, KC_SPH_EMF, [&] { k_sph_emf<float, true><<<nblk(D.NE), SPT, 0, S->s>>>(D, S->W32); });
        timed(S, KC_SPH_UPDATE_FACES, [&] {
          k_sph_update_faces<<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W32.EE, pin, S->phi, pout, a, b, S->dt, S->phif);
        });
        timed(S, KC_SPH_UPDATE_CELLS, [&] {
          k_sph_update_cells_mx<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W32, S->U, dUin, S->dU, (float)b, S->dt,
                                                                 last);
        });
      } else {
        // cells: stage input U1 (U^n at the first stage): out = a U^n + b (in - dt R)
        const double *Uin = st == 0 ? S->U : S->U1;
        double *Uout = last ? S->U : S->U1;
        if (prims) sph_prims(S, Uin, nullptr, pin, nullptr);
        timed(S, KC_SPH_FLUX, [&] {
          if (D.stellar) k_sph_flux<double, false, true><<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W64, pin, nullptr);
          else k_sph_flux<double, false><<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W64, pin, nullptr);
        });
        timed(S, KC_SPH_EMF, [&] { k_sph_emf<double, false><<<nblk(D.NE), SPT, 0, S->s>>>(D, S->W64); });
        timed(S, KC_SPH_UPDATE_FACES, [&] {
          k_sph_update_faces<<<nblk(D.NF), SPT, 0, S->s>>>(D, S->W64.EE, pin, S->phi, pout, a, b, S->dt, nullptr);
        });
        timed(S, KC_SPH_UPDATE_CELLS, [&] {
          k_sph_update_cells<<<nblk(D.ncell), SPT, 0, S->s>>>(D, S->W64, Uin, S->U, Uout, a, b, S->dt);
        });
      }
    }
  }
}
}  // namespace

extern "C" {

phl_status phl_sphere_step(phl_sphere *S, double dt, int nsteps) {
  if (!S || nsteps < 0 || !(dt == dt)) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_step: bad arguments");
  int done = 0;
  if (nsteps > 0 && S->cold) {   // a cold start's first step launches the network's guesses once
    sph_steps(S, dt, 1);
    done = 1;
  }
  if (S->use_graph && !S->prof.on && done < nsteps && sph_graph(S, dt)) {
    for (; done < nsteps; ++done) {
      const cudaError_t e = cudaGraphLaunch(S->gexec, S->s);
      if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_step: %s", cudaGetErrorString(e));
    }
  }
  sph_steps(S, dt, nsteps - done);
  S->steps += nsteps;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_sphere_step: %s", cudaGetErrorString(e));
  return PHL_OK;
}

phl_status phl_sphere_check(phl_sphere *S) {
  if (!S) return (phl_status)set_error(PHL_EINVAL, "phl_sphere_check: null sphere");
  return sph_flags(S);
}

}  // extern "C"
