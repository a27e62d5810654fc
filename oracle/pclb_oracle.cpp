// ============================================================================
// Oracle for the polar-coordinate finite-difference lattice Boltzmann step
// (Lin, Xu, Zhang, Li & Succi, "Polar coordinate lattice Boltzmann modeling
// of compressible flows").
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 restatement of
// the paper's method, written to be checked against the paper by eye.  Only
// the test suite, the smoke check and the benchmark's CPU-baseline leg may
// load it; the product (the CUDA library) never does, and the two share no
// code, headers or tables.
//
// What it computes, in the paper's order and notation:
//   * the discrete velocity model, Eq. (2), with N_k = 4 shells;
//   * the macroscopic moments rho, u, E, Eqs. (3)-(5);
//   * the weights F_k, Eqs. (11a), (11b), (12), and the equilibrium, Eq. (10);
//   * one time step of the combined scheme, Eq. (38): analytic relaxation,
//     Eq. (19), minus the Modified Warming-Beam terms, Eq. (28) with the switch
//     function S(eta) of Eq. (37), in r and in theta; and the variants the
//     paper compares: forward-Euler relaxation (Eq. 18), Warming-Beam
//     (Eq. 25), Lax-Wendroff and second-order upwind convection;
//   * the radial ghost nodes of Sec. II C 1 (Eq. 39, ghost f = f^eq) and the
//     azimuthal ghost nodes of Sec. II C 2 (Eq. 40, index rotation).
//   * the non-equilibrium manifestations of Sec. IV: the moments M_2, M_3,
//     M_{3,1}, M_{4,2} of f and their central counterparts M*_m (velocities
//     relative to the local flow velocity), and the departures
//     Delta_m = M_m(f - f^eq), Delta*_m = M*_m(f - f^eq);
//   * the vector-Jacobian product of that step (the adjoint step), by its
//     plain definition: forward-mode derivatives column by column, each
//     dotted with the cotangent.
//
// Readings where the paper is silent:
//   * velocity labels are fixed in Cartesian space: v_r = v.e_r(theta),
//     v_theta = v.e_theta(theta) at the node being updated;
//   * delta == 0 in Eq. (28): eta is undefined, the bracket times delta is
//     replaced by its limit C*delta (= 0); |eta| overflowing to infinity is
//     replaced by its limit;
//   * the derivative of |x| at x = 0 is taken as 0 (active-branch convention);
//   * ghost nodes: rho and T extrapolated by Eq. (39), applied twice for the
//     outer ghost layer; u extrapolated the same way (BC kind 0), prescribed
//     (kind 1), or everything prescribed (kind 2); f = f^eq there, or with
//     the flag 8 added to the kind, f^eq plus the non-equilibrium part
//     f - f^eq of the wall node.
//
// Parity pins for every function here live in tests/test_oracle_*.py.
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fopenmp -shared -fPIC.
// ============================================================================
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number (value, derivative), used only by the adjoint.
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
inline Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
inline Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
inline Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
inline Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
inline Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
inline Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
inline Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
inline Dual operator/(double a, Dual b) { return Dual(a) / b; }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
// A stored input value as the independent variable of a forward-mode sweep.
template <class T>
T seeded(double x);
template <>
inline double seeded<double>(double x) { return x; }
template <>
inline Dual seeded<Dual>(double x) { return Dual(x, 1.0); }
inline double sgn(double x) { return (x > 0) - (x < 0); }
inline double absval(double x) { return std::fabs(x); }
// |x| with d|x|/dx = sign(x), sign(0) = 0.
inline Dual absval(const Dual& x) { return {std::fabs(x.v), sgn(x.v) * x.d}; }

// ---------------------------------------------------------------------------
// Discrete velocity model, Eq. (2): v_ki = v_k (cos(2 pi (i-1)/N_i),
// sin(2 pi (i-1)/N_i)), k = 1..4, i = 1..N_i, plus the rest velocity v_0 = 0
// counted once.  Index q = 0 is the rest velocity, q = 1 + (k-1) N_i + (i-1).
// ---------------------------------------------------------------------------
struct Dvm {
  int n_dirs, Q;
  double speed[5];
  double B[5];
  std::vector<double> vx, vy;
  std::vector<int> shell, dir;  // shell k (0..4) and direction i (1..N_i; 0 for rest)
};

Dvm make_dvm(int n_dirs, const double* speeds, const double* B) {
  Dvm d;
  d.n_dirs = n_dirs;
  d.Q = 1 + 4 * n_dirs;
  for (int k = 0; k < 5; ++k) { d.speed[k] = speeds[k]; d.B[k] = B[k]; }
  d.vx.assign(d.Q, 0.0); d.vy.assign(d.Q, 0.0);
  d.shell.assign(d.Q, 0); d.dir.assign(d.Q, 0);
  for (int k = 1; k <= 4; ++k)
    for (int i = 1; i <= n_dirs; ++i) {
      int q = 1 + (k - 1) * n_dirs + (i - 1);
      double phi = 2.0 * M_PI * (i - 1) / n_dirs;
      d.vx[q] = speeds[k] * std::cos(phi);
      d.vy[q] = speeds[k] * std::sin(phi);
      d.shell[q] = k;
      d.dir[q] = i;
    }
  return d;
}

// mod{a, b} of Eq. (12).
int paper_mod(int a, int b) { return a <= b ? a : a - b; }

// Weights F_k(E), Eq. (11a) for k = 1..4 and Eq. (11b) for F_0.
template <class T>
void weights(const Dvm& d, T E, T F[5]) {
  for (int k = 1; k <= 4; ++k) {
    double vk2 = d.speed[k] * d.speed[k];
    double a = d.speed[paper_mod(k + 1, 4)] * d.speed[paper_mod(k + 1, 4)];
    double b = d.speed[paper_mod(k + 2, 4)] * d.speed[paper_mod(k + 2, 4)];
    double c = d.speed[paper_mod(k + 3, 4)] * d.speed[paper_mod(k + 3, 4)];
    T E2 = E * E, E3 = E2 * E, E4 = E3 * E;
    T num = d.B[4] * E4 + d.B[3] * (a + b + c) * E3 + d.B[2] * (a * b + b * c + c * a) * E2 +
            d.B[1] * (a * b * c) * E;
    double den = vk2 * (vk2 - a) * (vk2 - b) * (vk2 - c);
    F[k] = num / den;
  }
  F[0] = 1.0 - d.B[0] * (F[1] + F[2] + F[3] + F[4]);
}

// Equilibrium distribution, Eq. (10), for one node.
template <class T>
void feq_node(const Dvm& d, T rho, T ux, T uy, T E, T* feq) {
  T F[5];
  weights(d, E, F);
  T u2 = ux * ux + uy * uy;
  T a = 1.0 - u2 / (2.0 * E);
  for (int q = 0; q < d.Q; ++q) {
    T vu = d.vx[q] * ux + d.vy[q] * uy;  // v_{ki eps} u_eps
    T bracket = (1.0 - u2 / (2.0 * E) + u2 * u2 / (8.0 * E * E)) + (vu / E) * a +
                (vu * vu / (2.0 * E * E)) * a + vu * vu * vu / (6.0 * E * E * E) +
                vu * vu * vu * vu / (24.0 * E * E * E * E);
    feq[q] = rho * F[d.shell[q]] * bracket;
  }
}

// Macroscopic moments of one node, Eqs. (3)-(5): rho = sum f,
// rho u = sum f v, rho E = sum f |v - u|^2 / 2.  f[q * stride].
template <class T>
void moments_node(const Dvm& d, const T* f, long stride, T& rho, T& ux, T& uy, T& E) {
  T s0 = 0.0, sx = 0.0, sy = 0.0;
  for (int q = 0; q < d.Q; ++q) {
    T fq = f[q * stride];
    s0 += fq;
    sx += fq * d.vx[q];
    sy += fq * d.vy[q];
  }
  rho = s0;
  ux = sx / rho;
  uy = sy / rho;
  T se = 0.0;
  for (int q = 0; q < d.Q; ++q) {
    T cx = d.vx[q] - ux, cy = d.vy[q] - uy;
    se += 0.5 * f[q * stride] * (cx * cx + cy * cy);
  }
  E = se / rho;
}

// The Modified Warming-Beam increment of Eq. (28) for one node, i.e.
//   [C + C (1 - |C|) (1 - S(eta)) (1 - eta) / 2] * delta
// with delta and eta taken on the upwind side chosen by the sign of C
// (Eq. 27 / the definitions under Eq. 38) and S(eta) = (|eta| - 1)/(|eta| + 1)
// (Eq. 37).  Arguments are psi_{j-2} .. psi_{j+2}.
template <class T>
T mwb_increment(double C, T pm2, T pm1, T p0, T pp1, T pp2) {
  T delta, upstream;
  if (C >= 0) {
    delta = p0 - pm1;
    upstream = pm1 - pm2;
  } else {
    delta = pp1 - p0;
    upstream = pp2 - pp1;
  }
  if (val(delta) == 0.0) return C * delta;  // limit of the bracket times delta
  T eta = upstream / delta;
  if (!std::isfinite(val(eta)))  // |eta| -> infinity: (1-S)(1-eta) delta -> -2|delta| sign(upstream)
    return C * delta - C * (1.0 - std::fabs(C)) * absval(delta) * sgn(val(upstream));
  T S = (absval(eta) - 1.0) / (absval(eta) + 1.0);
  return (C + 0.5 * C * (1.0 - std::fabs(C)) * (1.0 - S) * (1.0 - eta)) * delta;
}

// The other convection schemes the paper compares (Sec. II B 3, Fig. 5), as
// the increment M with psi_j^{n+1} = psi_j^n - M; arguments psi_{j-2..j+2}.
// Warming-Beam, Eq. (25): second-order upwind differences in the Taylor
// expansion of Eq. (22).
template <class T>
T wb_increment(double C, T pm2, T pm1, T p0, T pp1, T pp2) {
  if (C >= 0) return C * (p0 - pm1) + 0.5 * C * (1.0 - C) * (p0 - 2.0 * pm1 + pm2);
  return C * (pp1 - p0) - 0.5 * C * (1.0 + C) * (p0 - 2.0 * pp1 + pp2);
}
// Lax-Wendroff: centred differences in the same Taylor expansion.
template <class T>
T lw_increment(double C, T pm2, T pm1, T p0, T pp1, T pp2) {
  (void)pm2;
  (void)pp2;
  return 0.5 * C * (pp1 - pm1) - 0.5 * C * C * (pp1 - 2.0 * p0 + pm1);
}
// Second-order upwind: a forward-Euler step with the derivative of Eq. (23).
template <class T>
T upwind2_increment(double C, T pm2, T pm1, T p0, T pp1, T pp2) {
  if (C >= 0) return 0.5 * C * (3.0 * p0 - 4.0 * pm1 + pm2);
  return -0.5 * C * (3.0 * p0 - 4.0 * pp1 + pp2);
}
template <class T>
T convection_increment(int scheme, double C, T pm2, T pm1, T p0, T pp1, T pp2) {
  switch (scheme) {
    case 1: return wb_increment(C, pm2, pm1, p0, pp1, pp2);
    case 2: return lw_increment(C, pm2, pm1, p0, pp1, pp2);
    case 3: return upwind2_increment(C, pm2, pm1, p0, pp1, pp2);
    default: return mwb_increment(C, pm2, pm1, p0, pp1, pp2);
  }
}

}  // namespace

// ============================================================================
// C interface (ctypes).
// ============================================================================
extern "C" {

typedef struct {
  int32_t n_r, n_theta;     // interior nodes in r and theta
  int32_t n_dirs, n_f;      // N_i directions; N_f sector periods (n_f == n_dirs: full circle)
  double r_in, r_out;       // R1, R2
  double speeds[5];         // v_0 .. v_4
  double B[5];              // B[n] = B_n of Table I (B[0] is the F_0 factor)
  double tau, dt;
  int32_t bc_kind[2];       // inner, outer: 0 extrapolate, 1 wall (u given), 2 all given (+8: ghost f - f^eq)
  const double* bc_values[2];  // [2 layers][4 fields rho,u_r,u_theta,T][n_theta]
  int32_t scheme;           // convection: 0 MWB (Eq. 28), 1 Warming-Beam, 2 Lax-Wendroff, 3 second-order upwind
  int32_t relaxation;       // 0 analytic exponential (Eq. 19), 1 forward Euler
} orc_problem;

enum { ORC_OK = 0, ORC_NONPHYS = 1, ORC_NONFINITE = 2, ORC_EINVAL = 4 };

}  // extern "C"

namespace {

// One time step of Eq. (38) with the boundary nodes of Sec. II C.
// f_in, f_out: [Q][n_theta][n_r].  Returns a status bitmask.
// Ghost nodes of one theta row at one wall, Sec. II C 1: macroscopic
// quantities from Eq. (39) (or prescribed), f = f^eq there.  fa, fb: the Q
// values at the wall node (i_r = 1 or N_r) and the next node inward; fe1,
// fe2: f at the adjacent and the outer ghost node.  With the non-equilibrium
// flag (kind & 8) the ghost nodes also carry the departure f - f^eq of the
// wall node (the non-equilibrium microscopic boundary of Sec. II C 1, in the
// form of the cited extrapolation scheme: the non-equilibrium part of the
// nearest fluid node is copied to the boundary).
template <class T>
int radial_ghost_layers(const orc_problem& P, const Dvm& d, int it, int side, const T* fa, const T* fb, T* fe1,
                        T* fe2) {
  const int NT = P.n_theta;
  const double dth = 2.0 * M_PI * P.n_f / (double(P.n_dirs) * NT);       // Sec. II C 2
  const double theta = (it + 1) * dth;
  const double c = std::cos(theta), s = std::sin(theta);
  T ra, uxa, uya, Ea, rb, uxb, uyb, Eb;
  moments_node(d, fa, 1, ra, uxa, uya, Ea);
  moments_node(d, fb, 1, rb, uxb, uyb, Eb);
  T rho1 = 2.0 * ra - rb, rho2 = 2.0 * rho1 - ra;   // Eq. (39), applied twice
  T E1 = 2.0 * Ea - Eb, E2 = 2.0 * E1 - Ea;         // "temperature in a similar way"
  T ux1 = 2.0 * uxa - uxb, ux2 = 2.0 * ux1 - uxa;
  T uy1 = 2.0 * uya - uyb, uy2 = 2.0 * uy1 - uya;
  const int kind = P.bc_kind[side] & 3;
  const bool neq = (P.bc_kind[side] & 8) != 0;
  const double* V = P.bc_values[side];
  auto given = [&](int layer, int field) { return V[((size_t)layer * 4 + field) * NT + it]; };
  if (kind == 1 || kind == 2) {  // prescribed polar velocity at the ghost nodes
    ux1 = T(given(0, 1) * c - given(0, 2) * s);
    uy1 = T(given(0, 1) * s + given(0, 2) * c);
    ux2 = T(given(1, 1) * c - given(1, 2) * s);
    uy2 = T(given(1, 1) * s + given(1, 2) * c);
  }
  if (kind == 2) {
    rho1 = T(given(0, 0)); E1 = T(given(0, 3));
    rho2 = T(given(1, 0)); E2 = T(given(1, 3));
  }
  int status = 0;
  if (!(val(rho1) > 0 && val(rho2) > 0 && val(E1) > 0 && val(E2) > 0)) status |= ORC_NONPHYS;
  feq_node(d, rho1, ux1, uy1, E1, fe1);
  feq_node(d, rho2, ux2, uy2, E2, fe2);
  if (neq) {
    std::vector<T> ea(d.Q);
    feq_node(d, ra, uxa, uya, Ea, ea.data());
    for (int q = 0; q < d.Q; ++q) {
      const T na = fa[q] - ea[q];
      fe1[q] = fe1[q] + na;
      fe2[q] = fe2[q] + na;
    }
  }
  return status;
}

// Label whose values fill the azimuthal ghost rows of label q, Eq. (40): the
// direction index rotated by N_f, for rows below the first (lo) and above the
// last (hi) interior row.
inline void azimuthal_labels(const orc_problem& P, const Dvm& d, int q, int& q_lo, int& q_hi) {
  q_lo = q_hi = q;
  if (d.shell[q] > 0) {
    int k = d.shell[q], i = d.dir[q];
    int i_lo = paper_mod(i + P.n_f, P.n_dirs);
    int i_hi = paper_mod(i - P.n_f + P.n_dirs, P.n_dirs);
    q_lo = 1 + (k - 1) * P.n_dirs + (i_lo - 1);
    q_hi = 1 + (k - 1) * P.n_dirs + (i_hi - 1);
  }
}

// Combined scheme, Eq. (38), at node (it, ir) (0-based interior indices).
// G(q, jt, jr) gives f with two ghost layers on every side (jt, jr from -2
// to N + 1).  Writes the Q updated values to out.
template <class T, class Get>
int update_node(const orc_problem& P, const Dvm& d, int it, int ir, Get G, T* out) {
  const int NR = P.n_r, NT = P.n_theta, Q = d.Q;
  const double dr = (P.r_out - P.r_in) / (NR - 1);                       // Sec. II C 1
  const double dth = 2.0 * M_PI * P.n_f / (double(P.n_dirs) * NT);       // Sec. II C 2
  // Eq. (19), or the forward-Euler step f + dt/tau (f^eq - f) of Eq. (18)
  const double decay = P.relaxation == 1 ? 1.0 - P.dt / P.tau : std::exp(-P.dt / P.tau);
  const double theta = (it + 1) * dth;
  const double c = std::cos(theta), s = std::sin(theta);
  const double r = P.r_in + ir * dr;
  int status = 0;
  std::vector<T> fc(Q), fe(Q);
  for (int q = 0; q < Q; ++q) fc[q] = G(q, it, ir);
  T rho, ux, uy, E;
  moments_node(d, fc.data(), 1, rho, ux, uy, E);
  if (!(val(rho) > 0 && val(E) > 0)) status |= ORC_NONPHYS;
  feq_node(d, rho, ux, uy, E, fe.data());
  for (int q = 0; q < Q; ++q) {
    const double v_r = d.vx[q] * c + d.vy[q] * s;
    const double v_t = -d.vx[q] * s + d.vy[q] * c;
    const double C_r = v_r * P.dt / dr;
    const double C_t = v_t * P.dt / (r * dth);
    T f = fc[q];
    T relax = fe[q] + (f - fe[q]) * decay;
    T term_r = convection_increment(P.scheme, C_r, G(q, it, ir - 2), G(q, it, ir - 1), f, G(q, it, ir + 1),
                                    G(q, it, ir + 2));
    T term_t = convection_increment(P.scheme, C_t, G(q, it - 2, ir), G(q, it - 1, ir), f, G(q, it + 1, ir),
                                    G(q, it + 2, ir));
    out[q] = relax - term_r - term_t;
    if (!std::isfinite(val(out[q]))) status |= ORC_NONFINITE;
  }
  return status;
}

template <class T>
int step_impl(const orc_problem& P, const Dvm& d, const T* f_in, T* f_out, bool parallel) {
  const int NR = P.n_r, NT = P.n_theta, Q = d.Q;

  // Extended array with two ghost layers on every side; corner ghosts are
  // never read by the axis-aligned stencils and stay NaN.
  const int ER = NR + 4, ET = NT + 4;
  std::vector<T> g((size_t)Q * ET * ER, T(std::numeric_limits<double>::quiet_NaN()));
  auto G = [&](int q, int it, int ir) -> T& {  // it, ir: 0-based interior index, ghosts -2,-1,N,N+1
    return g[((size_t)q * ET + (it + 2)) * ER + (ir + 2)];
  };
  for (int q = 0; q < Q; ++q)
    for (int it = 0; it < NT; ++it)
      for (int ir = 0; ir < NR; ++ir) G(q, it, ir) = f_in[((size_t)q * NT + it) * NR + ir];

  int status = 0;

  // (1) Radial ghost nodes, Sec. II C 1.
  {
    std::vector<T> fa(Q), fb(Q), fe1(Q), fe2(Q);
    for (int it = 0; it < NT; ++it)
      for (int side = 0; side < 2; ++side) {
        const int ia = side == 0 ? 0 : NR - 1;       // wall node i_r = 1 or N_r
        const int ib = side == 0 ? 1 : NR - 2;       // next node inward
        const int g1 = side == 0 ? -1 : NR;          // adjacent ghost (i_r = 0 or N_r + 1)
        const int g2 = side == 0 ? -2 : NR + 1;      // outer ghost (i_r = -1 or N_r + 2)
        for (int q = 0; q < Q; ++q) {
          fa[q] = G(q, it, ia);
          fb[q] = G(q, it, ib);
        }
        status |= radial_ghost_layers(P, d, it, side, fa.data(), fb.data(), fe1.data(), fe2.data());
        for (int q = 0; q < Q; ++q) {
          G(q, it, g1) = fe1[q];
          G(q, it, g2) = fe2[q];
        }
      }
  }

  // (2) Azimuthal ghost nodes, Eq. (40): copies of the rows at the other end
  //     of the period with the direction label rotated by N_f.
  for (int q = 0; q < Q; ++q) {
    int q_lo, q_hi;
    azimuthal_labels(P, d, q, q_lo, q_hi);
    for (int ir = 0; ir < NR; ++ir) {
      G(q, -2, ir) = G(q_lo, NT - 2, ir);
      G(q, -1, ir) = G(q_lo, NT - 1, ir);
      G(q, NT, ir) = G(q_hi, 0, ir);
      G(q, NT + 1, ir) = G(q_hi, 1, ir);
    }
  }

  // (3) Combined scheme, Eq. (38), at every node.
  auto Gv = [&](int q, int it, int ir) -> T { return G(q, it, ir); };
#pragma omp parallel for schedule(static) reduction(| : status) if (parallel)
  for (int it = 0; it < NT; ++it) {
    std::vector<T> out(Q);
    for (int ir = 0; ir < NR; ++ir) {
      status |= update_node(P, d, it, ir, Gv, out.data());
      for (int q = 0; q < Q; ++q) f_out[((size_t)q * NT + it) * NR + ir] = out[q];
    }
  }
  return status;
}

// The same step evaluated only at chosen nodes, reading f_in in place: the
// extended values the stencils need are formed on demand with exactly the
// operations of step_impl (wrapped rows with rotated labels; radial ghost
// layers of the rows that are read).  seed >= 0 marks one stored entry
// q * NT * NR + it * NR + ir whose derivative is 1 (T = Dual), for the
// node-local adjoint below.
template <class T>
int step_nodes_impl(const orc_problem& P, const Dvm& d, const double* f_in, long seed, int n, const int32_t* it_list,
                    const int32_t* ir_list, T* out) {
  const int NR = P.n_r, NT = P.n_theta, Q = d.Q;
  std::vector<int> qlo(Q), qhi(Q);
  for (int q = 0; q < Q; ++q) azimuthal_labels(P, d, q, qlo[q], qhi[q]);
  auto stored = [&](int q, int it, int ir) -> T {   // interior entry, it in [0, NT)
    const long idx = ((long)q * NT + it) * NR + ir;
    T v = T(f_in[idx]);
    if (idx == seed) v = seeded<T>(f_in[idx]);
    return v;
  };
  int status = 0;
  std::vector<T> fa(Q), fb(Q), fe1(Q), fe2(Q);
  // radial ghost layers of row `it` at `side`, recomputed when first needed
  std::vector<std::vector<T>> gcache;
  std::vector<long> gkey;
  auto ghost = [&](int it, int side, int layer, int q) -> T {
    const long key = ((long)it * 2 + side);
    for (size_t j = 0; j < gkey.size(); ++j)
      if (gkey[j] == key) return gcache[j][(size_t)layer * Q + q];
    const int ia = side == 0 ? 0 : NR - 1, ib = side == 0 ? 1 : NR - 2;
    for (int p = 0; p < Q; ++p) {
      fa[p] = stored(p, it, ia);
      fb[p] = stored(p, it, ib);
    }
    status |= radial_ghost_layers(P, d, it, side, fa.data(), fb.data(), fe1.data(), fe2.data());
    std::vector<T> both(2 * Q);
    for (int p = 0; p < Q; ++p) {
      both[p] = fe1[p];
      both[Q + p] = fe2[p];
    }
    gkey.push_back(key);
    gcache.push_back(both);
    return gcache.back()[(size_t)layer * Q + q];
  };
  auto G = [&](int q, int it, int ir) -> T {
    if (it < 0 || it >= NT) {                     // azimuthal ghost rows, Eq. (40)
      if (ir < 0 || ir >= NR) return T(std::numeric_limits<double>::quiet_NaN());   // corner
      return it < 0 ? stored(qlo[q], it + NT, ir) : stored(qhi[q], it - NT, ir);
    }
    if (ir < 0) return ghost(it, 0, ir == -1 ? 0 : 1, q);
    if (ir >= NR) return ghost(it, 1, ir == NR ? 0 : 1, q);
    return stored(q, it, ir);
  };
  for (int j = 0; j < n; ++j) status |= update_node(P, d, it_list[j], ir_list[j], G, out + (size_t)j * Q);
  return status;
}

bool valid(const orc_problem* P) {
  if (!P) return false;
  if (P->n_r < 3 || P->n_theta < 2) return false;
  if (P->n_dirs < 1 || P->n_f < 1 || P->n_f > P->n_dirs) return false;
  if (!(P->r_out > P->r_in) || !(P->r_in > 0) || !(P->tau > 0) || !(P->dt > 0)) return false;
  if (P->scheme < 0 || P->scheme > 3 || P->relaxation < 0 || P->relaxation > 1) return false;
  for (int s = 0; s < 2; ++s) {
    if ((P->bc_kind[s] & ~(3 | 8)) != 0 || (P->bc_kind[s] & 3) == 3) return false;
    if ((P->bc_kind[s] & 3) != 0 && P->bc_values[s] == nullptr) return false;
  }
  return true;
}

// f = f^eq of the fields (initial equilibrium); fields [n_theta][n_r] with
// polar velocity components, f [Q][n_theta][n_r].
template <class T>
int set_state_impl(const orc_problem& P, const Dvm& d, const T* rho, const T* u_r, const T* u_t, const T* E,
                   T* f) {
  const int NR = P.n_r, NT = P.n_theta;
  const double dth = 2.0 * M_PI * P.n_f / (double(P.n_dirs) * NT);
  int status = 0;
#pragma omp parallel for schedule(static) reduction(| : status)
  for (int it = 0; it < NT; ++it) {
    std::vector<T> fe(d.Q);
    const double th = (it + 1) * dth, c = std::cos(th), s = std::sin(th);
    for (int ir = 0; ir < NR; ++ir) {
      size_t n = (size_t)it * NR + ir;
      if (!(val(rho[n]) > 0 && val(E[n]) > 0)) status |= ORC_NONPHYS;
      T ux = u_r[n] * c - u_t[n] * s, uy = u_r[n] * s + u_t[n] * c;
      feq_node(d, rho[n], ux, uy, E[n], fe.data());  // E = T / (gamma - 1), gamma = 2
      for (int q = 0; q < d.Q; ++q) f[((size_t)q * NT + it) * NR + ir] = fe[q];
    }
  }
  return status;
}

// rho, u_r, u_theta, T of every node (Eqs. 3-5, polar components).
template <class T>
void fields_impl(const orc_problem& P, const Dvm& d, const T* f, T* rho, T* u_r, T* u_t, T* E) {
  const int NR = P.n_r, NT = P.n_theta;
  const double dth = 2.0 * M_PI * P.n_f / (double(P.n_dirs) * NT);
  for (int it = 0; it < NT; ++it) {
    const double th = (it + 1) * dth, c = std::cos(th), s = std::sin(th);
    for (int ir = 0; ir < NR; ++ir) {
      size_t n = (size_t)it * NR + ir;
      T r_, ux, uy, e_;
      moments_node(d, f + n, (long)NT * NR, r_, ux, uy, e_);
      if (rho) rho[n] = r_;
      if (u_r) u_r[n] = ux * c + uy * s;
      if (u_t) u_t[n] = -ux * s + uy * c;
      if (E) E[n] = e_;
    }
  }
}

}  // namespace

extern "C" {

int orc_q(int n_dirs) { return 1 + 4 * n_dirs; }

void orc_dvm(int n_dirs, const double* speeds, double* vx, double* vy, int32_t* shell) {
  const double B[5] = {0, 0, 0, 0, 0};
  Dvm d = make_dvm(n_dirs, speeds, B);
  for (int q = 0; q < d.Q; ++q) { vx[q] = d.vx[q]; vy[q] = d.vy[q]; shell[q] = d.shell[q]; }
}

void orc_weights(int n_dirs, const double* speeds, const double* B, double E, double* F) {
  Dvm d = make_dvm(n_dirs, speeds, B);
  weights(d, E, F);
}

void orc_feq(int n_dirs, const double* speeds, const double* B, double rho, double ux, double uy,
             double E, double* feq) {
  Dvm d = make_dvm(n_dirs, speeds, B);
  feq_node(d, rho, ux, uy, E, feq);
}

// out = (rho, u_x, u_y, E)
void orc_moments(int n_dirs, const double* speeds, const double* f, double* out) {
  const double B[5] = {0, 0, 0, 0, 0};
  Dvm d = make_dvm(n_dirs, speeds, B);
  moments_node(d, f, 1, out[0], out[1], out[2], out[3]);
}

double orc_scheme_increment(int scheme, double C, double pm2, double pm1, double p0, double pp1, double pp2) {
  return convection_increment(scheme, C, pm2, pm1, p0, pp1, pp2);
}

double orc_mwb_increment(double C, double pm2, double pm1, double p0, double pp1, double pp2) {
  return mwb_increment(C, pm2, pm1, p0, pp1, pp2);
}

// The bare MWB scheme, Eq. (28), on a periodic 1-D array with constant C.
void orc_mwb_1d(int n, const double* psi, double C, double* out) {
  for (int j = 0; j < n; ++j) {
    auto at = [&](int k) { return psi[((k % n) + n) % n]; };
    out[j] = psi[j] - mwb_increment(C, at(j - 2), at(j - 1), at(j), at(j + 1), at(j + 2));
  }
}

// f = f^eq of the given fields (initially in equilibrium).  Fields
// [n_theta][n_r], polar velocity components; f: [Q][n_theta][n_r].
int orc_set_state(const orc_problem* P, const double* rho, const double* u_r, const double* u_t,
                  const double* T, double* f) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  return set_state_impl<double>(*P, d, rho, u_r, u_t, T, f);
}

// Directional derivative of f^eq(fields): df = d f^eq / d fields . dfields.
// fields / dfields: 4 arrays each [n_theta][n_r] (rho, u_r, u_theta, T).
int orc_set_state_jvp(const orc_problem* P, const double* const* fields, const double* const* dfields,
                      double* df) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const size_t N = (size_t)P->n_r * P->n_theta;
  std::vector<Dual> x[4];
  for (int k = 0; k < 4; ++k) {
    x[k].resize(N);
    for (size_t n = 0; n < N; ++n) x[k][n] = Dual(fields[k][n], dfields[k][n]);
  }
  std::vector<Dual> y((size_t)d.Q * N);
  int st = set_state_impl<Dual>(*P, d, x[0].data(), x[1].data(), x[2].data(), x[3].data(), y.data());
  for (size_t i = 0; i < y.size(); ++i) df[i] = y[i].d;
  return st;
}

// rho, u_r, u_theta, T of every node from f (any output may be NULL).
int orc_fields(const orc_problem* P, const double* f, double* rho, double* u_r, double* u_t,
               double* T) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  fields_impl<double>(*P, d, f, rho, u_r, u_t, T);
  return 0;
}

// Directional derivative of the fields: dfields[k] = d field_k / d f . df.
int orc_fields_jvp(const orc_problem* P, const double* f, const double* df, double* const* dfields) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const size_t N = (size_t)P->n_r * P->n_theta;
  std::vector<Dual> x((size_t)d.Q * N), o[4];
  for (size_t i = 0; i < x.size(); ++i) x[i] = Dual(f[i], df[i]);
  for (int k = 0; k < 4; ++k) o[k].resize(N);
  fields_impl<Dual>(*P, d, x.data(), o[0].data(), o[1].data(), o[2].data(), o[3].data());
  for (int k = 0; k < 4; ++k)
    for (size_t n = 0; n < N; ++n) dfields[k][n] = o[k][n].d;
  return 0;
}

// Global integrals with the polar area element r dr dtheta:
// out = (mass, x-momentum, y-momentum, total energy, min rho, min T).
int orc_diagnostics(const orc_problem* P, const double* f, double* out) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const int NR = P->n_r, NT = P->n_theta;
  const double dr = (P->r_out - P->r_in) / (NR - 1);
  const double dth = 2.0 * M_PI * P->n_f / (double(P->n_dirs) * NT);
  double m = 0, jx = 0, jy = 0, e = 0, rmin = INFINITY, tmin = INFINITY;
  for (int it = 0; it < NT; ++it)
    for (int ir = 0; ir < NR; ++ir) {
      size_t n = (size_t)it * NR + ir;
      double rho, ux, uy, E;
      moments_node(d, f + n, (long)NT * NR, rho, ux, uy, E);
      double w = (P->r_in + ir * dr) * dr * dth;
      m += w * rho;
      jx += w * rho * ux;
      jy += w * rho * uy;
      e += w * rho * (E + 0.5 * (ux * ux + uy * uy));
      rmin = std::fmin(rmin, rho);
      tmin = std::fmin(tmin, E);
    }
  out[0] = m; out[1] = jx; out[2] = jy; out[3] = e; out[4] = rmin; out[5] = tmin;
  return 0;
}

// Non-equilibrium manifestations, Sec. IV.  For weights w_q (f, or f - f^eq)
// and velocities c_q (v_q, or v_q - u for the central moments), in polar
// components at the node (c_r = c . e_r, c_theta = c . e_theta):
//   M_2     = sum w c c                 -> rr, r theta, theta theta
//   M_3     = sum w c c c               -> rrr, rr theta, r theta theta, theta theta theta
//   M_{3,1} = sum w (c . c / 2) c       -> r, theta
//   M_{4,2} = sum w (c . c / 2) c c     -> rr, r theta, theta theta
// Group g (bit 0: M_m(f), bit 1: Delta_m, bit 2: M*_m(f), bit 3: Delta*_m)
// fills 12 fields [12][n_theta][n_r] of out, groups in bit order.
int orc_noneq(const orc_problem* P, const double* f, int groups, double* out) {
  if (!valid(P) || groups <= 0 || groups > 15) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const int NR = P->n_r, NT = P->n_theta, Q = d.Q;
  const double dth = 2.0 * M_PI * P->n_f / (double(P->n_dirs) * NT);
  const size_t plane = (size_t)NT * NR;
  int status = 0;
#pragma omp parallel for schedule(static) reduction(| : status)
  for (int it = 0; it < NT; ++it) {
    const double theta = (it + 1) * dth;
    const double cs = std::cos(theta), sn = std::sin(theta);
    std::vector<double> fe(Q);
    for (int ir = 0; ir < NR; ++ir) {
      const size_t n = (size_t)it * NR + ir;
      double rho, ux, uy, E;
      moments_node(d, f + n, (long)plane, rho, ux, uy, E);
      if (!(rho > 0 && E > 0)) status |= ORC_NONPHYS;
      feq_node(d, rho, ux, uy, E, fe.data());
      const double u_r = ux * cs + uy * sn, u_t = -ux * sn + uy * cs;
      int slot = 0;
      for (int g = 0; g < 4; ++g) {
        if (!(groups & (1 << g))) continue;
        const bool departure = g == 1 || g == 3, central = g >= 2;
        double m[12] = {0};
        for (int q = 0; q < Q; ++q) {
          const double w = departure ? f[q * plane + n] - fe[q] : f[q * plane + n];
          double cr = d.vx[q] * cs + d.vy[q] * sn, ct = -d.vx[q] * sn + d.vy[q] * cs;
          if (central) {
            cr -= u_r;
            ct -= u_t;
          }
          const double h = 0.5 * (cr * cr + ct * ct);
          m[0] += w * cr * cr;
          m[1] += w * cr * ct;
          m[2] += w * ct * ct;
          m[3] += w * cr * cr * cr;
          m[4] += w * cr * cr * ct;
          m[5] += w * cr * ct * ct;
          m[6] += w * ct * ct * ct;
          m[7] += w * h * cr;
          m[8] += w * h * ct;
          m[9] += w * h * cr * cr;
          m[10] += w * h * cr * ct;
          m[11] += w * h * ct * ct;
        }
        for (int c = 0; c < 12; ++c) out[((size_t)(slot * 12 + c)) * plane + n] = m[c];
        ++slot;
      }
    }
  }
  return status;
}

// One step of Eq. (38).  f_in, f_out: [Q][n_theta][n_r].
int orc_step(const orc_problem* P, const double* f_in, double* f_out, int parallel) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  return step_impl<double>(*P, d, f_in, f_out, parallel != 0);
}

// n steps; f is updated in place.
int orc_run(const orc_problem* P, double* f, int n, int parallel) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  size_t N = (size_t)d.Q * P->n_theta * P->n_r;
  std::vector<double> tmp(N);
  int status = 0;
  for (int s = 0; s < n; ++s) {
    status |= step_impl<double>(*P, d, f, tmp.data(), parallel != 0);
    std::memcpy(f, tmp.data(), N * sizeof(double));
  }
  return status;
}

// Directional derivative of one step: df_out = J(f) df.
int orc_step_jvp(const orc_problem* P, const double* f, const double* df, double* df_out) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  size_t N = (size_t)d.Q * P->n_theta * P->n_r;
  std::vector<Dual> x(N), y(N);
  for (size_t i = 0; i < N; ++i) x[i] = Dual(f[i], df[i]);
  int st = step_impl<Dual>(*P, d, x.data(), y.data(), false);
  for (size_t i = 0; i < N; ++i) df_out[i] = y[i].d;
  return st;
}

// Adjoint (vector-Jacobian product) of one step: lam_n = J(f_n)^T lam_np1,
// computed by its definition, one forward-mode column per input entry:
// lam_n[j] = < lam_np1, J e_j >.  Cost O(N^2): small grids only.
int orc_adjoint_step(const orc_problem* P, const double* f_n, const double* lam_np1,
                     double* lam_n) {
  if (!valid(P)) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const long N = (long)d.Q * P->n_theta * P->n_r;
  int status = 0;
#pragma omp parallel reduction(| : status)
  {
    std::vector<Dual> x(N), y(N);
#pragma omp for schedule(dynamic, 16)
    for (long j = 0; j < N; ++j) {
      for (long i = 0; i < N; ++i) x[i] = Dual(f_n[i], i == j ? 1.0 : 0.0);
      status |= step_impl<Dual>(*P, d, x.data(), y.data(), false);
      double acc = 0.0;
      for (long i = 0; i < N; ++i) acc += lam_np1[i] * y[i].d;
      lam_n[j] = acc;
    }
  }
  return status;
}

// f^{n+1} at chosen nodes only: out[j * Q + q] for the node (it[j], ir[j])
// (0-based), from the whole f^n.  Same operations as orc_step.
int orc_step_nodes(const orc_problem* P, const double* f_in, int n, const int32_t* it, const int32_t* ir,
                   double* out) {
  if (!valid(P)) return ORC_EINVAL;
  for (int j = 0; j < n; ++j)
    if (it[j] < 0 || it[j] >= P->n_theta || ir[j] < 0 || ir[j] >= P->n_r) return ORC_EINVAL;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  return step_nodes_impl<double>(*P, d, f_in, -1, n, it, ir, out);
}

// Chosen entries of the adjoint step, lam^n_q(it, ir) = sum over every output
// (q', node) of lam^{n+1}_q'(node) d f^{n+1}_q'(node) / d f^n_q(it, ir), by
// its definition: one forward-mode sweep seeded at the entry, over the nodes
// whose update can read it (the same theta row within two radial nodes, the
// same radius within two rows, azimuthal rows wrapped).
int orc_adjoint_entries(const orc_problem* P, const double* f_n, const double* lam_np1, int n, const int32_t* q,
                        const int32_t* it, const int32_t* ir, double* out) {
  if (!valid(P)) return ORC_EINVAL;
  const int NR = P->n_r, NT = P->n_theta;
  Dvm d = make_dvm(P->n_dirs, P->speeds, P->B);
  const int Q = d.Q;
  for (int j = 0; j < n; ++j)
    if (q[j] < 0 || q[j] >= Q || it[j] < 0 || it[j] >= NT || ir[j] < 0 || ir[j] >= NR) return ORC_EINVAL;
  int status = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : status)
  for (int j = 0; j < n; ++j) {
    std::vector<int32_t> nt, nr;
    auto add = [&](int t, int r) {
      t = ((t % NT) + NT) % NT;
      for (size_t m = 0; m < nt.size(); ++m)
        if (nt[m] == t && nr[m] == r) return;
      nt.push_back(t);
      nr.push_back(r);
    };
    for (int a = -2; a <= 2; ++a) add(it[j] + a, ir[j]);
    for (int b = -2; b <= 2; ++b)
      if (ir[j] + b >= 0 && ir[j] + b < NR) add(it[j], ir[j] + b);
    const long seed = ((long)q[j] * NT + it[j]) * NR + ir[j];
    std::vector<Dual> y(nt.size() * Q);
    status |= step_nodes_impl<Dual>(*P, d, f_n, seed, (int)nt.size(), nt.data(), nr.data(), y.data());
    double acc = 0.0;
    for (size_t m = 0; m < nt.size(); ++m)
      for (int p = 0; p < Q; ++p) acc += lam_np1[((size_t)p * NT + nt[m]) * NR + nr[m]] * y[m * Q + p].d;
    out[j] = acc;
  }
  return status;
}

}  // extern "C"
