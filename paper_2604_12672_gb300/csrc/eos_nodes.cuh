// eos_nodes.cuh -- node values of the stellar EOS table: the Helmholtz
// free-energy density of the electron-positron gas and the eight derivatives
// a biquintic Hermite interpolant needs (Sect. 2.2), from the generalised
// Fermi-Dirac integrals by quadrature.  Host and device (the table is built
// on the device; the host copy serves the library's own CPU checks).
//
// Variables: x = ln n_e (net electron density), y = ln T, b = kT / m_e c^2,
// xi = kinetic energy / m_e c^2 and psi = eta b (Fermi kinetic energy):
//   n = K_n [G_1/2 + G_3/2](psi) - K_n [G_1/2 + G_3/2](psi+),
//   P = K_p [G_3/2 + G_5/2 / 2](psi) + K_p [...](psi+),   psi+ = -psi - 2,
//   G_k(psi, y) = int xi^k sqrt(1 + xi/2) F((xi - psi) / b) dxi,  F(u) = 1/(e^u + 1).
// With u = (xi - psi)/b, d/dpsi acts on F(u) as -F'/b and d/dy (fixed psi)
// as -u F' (b = b0 e^(y - y0)), so every partial of G is a combination of
//   J[p][i] = int xi^k sqrt(1 + xi/2) u^i F^(p)(u) dxi.
// Thermodynamics fixes the rest: P_psi = m_e c^2 n (Gibbs-Duhem at fixed T),
// hence with f = n m_e c^2 psi - P
//   f_x = m c^2 n psi,        f_xx = m c^2 n (psi + psi_x),
//   f_y = -P_y,               f_yy = -(m c^2 N_y psi_y + P_yy),
//   f_xy = m c^2 n psi_y,     f_xxy = m c^2 n (psi_y + psi_xy),
//   f_xyy = m c^2 n psi_yy,   f_xxyy = m c^2 n (psi_yy + psi_xyy),
// where psi(x, y) solves N(psi, y) = e^x and its derivatives follow by
// implicit differentiation (N_psi psi_x = n, N_psi psi_y = -N_y, ...).
#pragma once
#include <math.h>

namespace phl {
namespace eosn {

constexpr double KB = 1.380649e-16;       // CODATA 2018 (CGS)
constexpr double MEC2 = 8.1871057769e-7;
constexpr double PI_D = 3.14159265358979323846;
constexpr int GLN = 32;                   // Gauss-Legendre order of the panels
constexpr int NQ = 9;                     // f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy

// Panel edges (in units of kT) around the Fermi edge x = max(eta, 0): the
// Fermi factor changes by at most e^20 across a panel and is below e^-50
// before the first edge.
__host__ __device__ __forceinline__ double panel_offset(int k) {
  const double off[14] = {-50.0, -30.0, -16.0, -8.0, -4.0, -1.5, 0.0, 1.5, 4.0, 8.0, 16.0, 30.0, 50.0, 110.0};
  return off[k];
}

// F_1/2, F_3/2, F_5/2, dF_{1/2,3/2}/deta, dF_{1/2,3/2}/db of one species at
// (eta, b): the integrals the neutrality root needs.  x = s^2.
__host__ __device__ inline void fd_integrals(double eta, double b, const double *glx, const double *glw, double *F) {
  for (int q = 0; q < 7; ++q) F[q] = 0.0;
  const double base = fmax(eta, 0.0);
  double a = 0.0;
  for (int k = 0; k < 14; ++k) {
    const double xe = base + panel_offset(k);
    if (!(xe > 0.0)) continue;
    const double c = sqrt(xe);
    if (!(c > a)) continue;
    const double hm = 0.5 * (c - a), cm = 0.5 * (c + a);
    for (int g = 0; g < GLN; ++g) {
      const double s = cm + hm * glx[g];
      const double wgt = 2.0 * s * hm * glw[g];   // dx = 2 s ds
      const double x = s * s, u = x - eta;
      const double z = exp(-fabs(u));
      const double fermi = u > 0.0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
      const double fder = z / ((1.0 + z) * (1.0 + z));   // -F'(u) = F (1 - F)
      const double S = sqrt(1.0 + 0.5 * b * x);
      const double x12 = s, x32 = x * s, x52 = x * x * s;
      F[0] += wgt * x12 * S * fermi;
      F[1] += wgt * x32 * S * fermi;
      F[2] += wgt * x52 * S * fermi;
      F[3] += wgt * x12 * S * fder;
      F[4] += wgt * x32 * S * fder;
      F[5] += wgt * x32 * fermi / (4.0 * S);
      F[6] += wgt * x52 * fermi / (4.0 * S);
    }
    a = c;
  }
}

struct SpeciesN { double n, n_eta; };

__host__ __device__ inline SpeciesN species_n(double eta, double b, double lam3, const double *glx, const double *glw) {
  double F[7];
  fd_integrals(eta, b, glx, glw, F);
  const double Kn = 8.0 * PI_D * sqrt(2.0) * lam3;
  const double b32 = b * sqrt(b);
  return SpeciesN{Kn * b32 * (F[0] + b * F[1]), Kn * b32 * (F[3] + b * F[4])};
}

// Moments of one species at its eta: J[k][m] with k = xi^(1/2), xi^(3/2),
// xi^(5/2) weights and m the (p, i) pairs (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
// (3,0) (3,1) (3,2) of u^i F^(p)(u).  F' = -g, F'' = g t, F''' = 2 g^2 - g t^2
// with g = F (1 - F), t = 1 - 2 F.
enum { J00 = 0, J10, J11, J20, J21, J22, J30, J31, J32, NJ };
__host__ __device__ inline void moments(double eta, double b, const double *glx, const double *glw, double J[3][NJ]) {
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < NJ; ++m) J[k][m] = 0.0;
  const double base = fmax(eta, 0.0);
  double a = 0.0;
  for (int k = 0; k < 14; ++k) {
    const double xe = base + panel_offset(k);
    if (!(xe > 0.0)) continue;
    const double c = sqrt(xe);
    if (!(c > a)) continue;
    const double hm = 0.5 * (c - a), cm = 0.5 * (c + a);
    for (int g = 0; g < GLN; ++g) {
      const double s = cm + hm * glx[g];
      const double x = s * s, u = x - eta;
      const double wgt = b * 2.0 * s * hm * glw[g];   // dxi = b dx
      const double z = exp(-fabs(u));
      const double F = u > 0.0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
      const double gg = z / ((1.0 + z) * (1.0 + z));
      const double t = u > 0.0 ? (1.0 - z) / (1.0 + z) : (z - 1.0) / (1.0 + z);
      const double F1 = -gg, F2 = gg * t, F3 = 2.0 * gg * gg - gg * t * t;
      const double xi = b * x, sxi = sqrt(xi), S = sqrt(1.0 + 0.5 * xi);
      const double w[3] = {wgt * sxi * S, wgt * xi * sxi * S, wgt * xi * xi * sxi * S};
      const double u2 = u * u;
      for (int q = 0; q < 3; ++q) {
        J[q][J00] += w[q] * F;
        J[q][J10] += w[q] * F1;
        J[q][J11] += w[q] * u * F1;
        J[q][J20] += w[q] * F2;
        J[q][J21] += w[q] * u * F2;
        J[q][J22] += w[q] * u2 * F2;
        J[q][J30] += w[q] * F3;
        J[q][J31] += w[q] * u * F3;
        J[q][J32] += w[q] * u2 * F3;
      }
    }
    a = c;
  }
}

// Partials of H = G_a + c G_b (one species) in (psi, y) from its moments.
struct HP { double v, p, pp, ppp, y, yy, py, ppy, pyy; };
__host__ __device__ inline HP h_partials(const double J[3][NJ], int ka, int kb, double cb, double b) {
  double m[NJ];
  for (int q = 0; q < NJ; ++q) m[q] = J[ka][q] + cb * J[kb][q];
  const double ib = 1.0 / b;
  HP h;
  h.v = m[J00];
  h.p = -ib * m[J10];
  h.pp = ib * ib * m[J20];
  h.ppp = -ib * ib * ib * m[J30];
  h.y = -m[J11];
  h.yy = m[J11] + m[J22];
  h.py = ib * (m[J10] + m[J21]);
  h.ppy = -ib * ib * (2.0 * m[J20] + m[J31]);
  h.pyy = -ib * (m[J10] + 3.0 * m[J21] + m[J32]);
  return h;
}

// The NQ node values at net density ne and temperature T (lam3 = (m_e c/h)^3);
// false if the neutrality root was not found.
__host__ __device__ inline bool node_values(double ne, double T, double lam3, const double *glx, const double *glw,
                                            double *o) {
  const double b = KB * T / MEC2;
  const double Kn = 8.0 * PI_D * sqrt(2.0) * lam3;
  const double Kp = (2.0 / 3.0) * Kn * MEC2;
  // charge neutrality n-(eta) - n+(-eta - 2/b) = ne: bracketed Newton
  const double xf = cbrt(3.0 * ne / (8.0 * PI_D * lam3));
  double eta = fmax(log(ne / (Kn * b * sqrt(b) * 0.886226925452758)), (sqrt(1.0 + xf * xf) - 1.0) / b);
  double lo = -700.0, hi = 1e7;
  bool ok = false;
  for (int it = 0; it < 200; ++it) {
    const SpeciesN m = species_n(eta, b, lam3, glx, glw), p = species_n(-eta - 2.0 / b, b, lam3, glx, glw);
    const double r = m.n - p.n - ne;
    if (r > 0.0) hi = eta; else lo = eta;
    double en = eta - r / (m.n_eta + p.n_eta);
    if (!(en > lo && en < hi)) en = 0.5 * (lo + hi);
    const bool done = fabs(en - eta) <= 1e-15 * (fabs(eta) + 1.0) || hi - lo < 1e-14 * (fabs(eta) + 1.0);
    eta = en;
    if (done) { ok = true; break; }
  }
  if (!ok) return false;
  const double psi = eta * b;
  double Jm[3][NJ], Jp[3][NJ];
  moments(eta, b, glx, glw, Jm);
  moments(-eta - 2.0 / b, b, glx, glw, Jp);
  // number-density part H = G_1/2 + G_3/2 and pressure part G_3/2 + G_5/2 / 2
  const HP Hm = h_partials(Jm, 0, 1, 1.0, b), Hp = h_partials(Jp, 0, 1, 1.0, b);
  const HP Qm = h_partials(Jm, 1, 2, 0.5, b), Qp = h_partials(Jp, 1, 2, 0.5, b);
  // N = Kn [H(psi) - H(-psi - 2)]: odd psi-derivatives of the positron term add
  const double Np = Kn * (Hm.p + Hp.p), Npp = Kn * (Hm.pp - Hp.pp), Nppp = Kn * (Hm.ppp + Hp.ppp);
  const double Ny = Kn * (Hm.y - Hp.y), Nyy = Kn * (Hm.yy - Hp.yy), Npy = Kn * (Hm.py + Hp.py);
  const double Nppy = Kn * (Hm.ppy - Hp.ppy), Npyy = Kn * (Hm.pyy + Hp.pyy);
  const double P = Kp * (Qm.v + Qp.v), Py = Kp * (Qm.y + Qp.y), Pyy = Kp * (Qm.yy + Qp.yy);
  // psi(x, y) from N(psi, y) = e^x
  const double px = ne / Np;
  const double py = -Ny / Np;
  const double A = Npp * py + Npy;                      // d(N_psi)/dy along the root
  const double pxy = -px * A / Np;
  const double pyy = -(Npp * py * py + 2.0 * Npy * py + Nyy) / Np;
  const double dA = Nppp * py * py + 2.0 * Nppy * py + Npp * pyy + Npyy;
  const double pxyy = -(px * dA + 2.0 * A * pxy) / Np;
  const double mn = MEC2 * ne;
  o[0] = mn * psi - P;               // f
  o[1] = mn * psi;                   // f_x
  o[2] = -Py;                        // f_y
  o[3] = mn * (psi + px);            // f_xx
  o[4] = -(MEC2 * Ny * py + Pyy);    // f_yy
  o[5] = mn * py;                    // f_xy
  o[6] = mn * (py + pxy);            // f_xxy
  o[7] = mn * pyy;                   // f_xyy
  o[8] = mn * (pyy + pxyy);          // f_xxyy
  return true;
}

}  // namespace eosn
}  // namespace phl
