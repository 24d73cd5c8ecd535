// FP64 CPU oracle of the Partially Saturated Cells Method (PSM) lattice Boltzmann
// step with moving-geometry remapping (arXiv 2502.20049, Sec. 2.1 and Sec. 3).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct
// restatement of the method that the CUDA library is checked against.  Only the
// test suite, the smoke check and the CPU-baseline leg of the benchmark load it.
// It shares no code, header, table or constant with the CUDA library.
//
// Conventions (readings of the paper, each restated where it is used):
//   * lattice units, dx = dt = 1, c_s^2 = 1/3;
//   * PDF array f[i][z][y][x] in natural (pull-streamed, pre-collision) form,
//     direction order of THIS file: lexicographic in (cz, cy, cx) over {-1,0,1}^3;
//   * one time step n = remap (Sec. 3) -> per-cell collision Eq. 4 with
//     Eq. 2/TRT/cumulant, Eq. 7-9, weighting Eq. 5/6 -> force/torque Eq. 10/11 ->
//     streaming Eq. 1 with periodic x/y and either periodic z or equilibrium
//     ghost planes in z;
//   * all arithmetic in double (or Dual<double> for the tangent-linear model);
//     the remap's body-frame transform and sub-cell decision are double
//     operations in the order written, each rounded on its own (the file is
//     compiled without floating-point contraction; the paper states no
//     precision for them).
//
// The scalar type is a template parameter so that the same code, run on
// forward-mode dual numbers, gives exact directional derivatives (tangent-linear
// model) of the force/torque series with respect to a per-cell fraction
// perturbation, the angular velocity and the inflow velocity.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual number (value + one tangent).
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline double tan_of(double) { return 0.0; }
inline double tan_of(const Dual& a) { return a.d; }

// ---------------------------------------------------------------------------
// Lattices D3Q19 and D3Q27 (standard velocity sets; the paper names them in
// Sec. 2.2 without tables).  Weights by |c|^2:
//   D3Q19: 0 -> 1/3, 1 -> 1/18, 2 -> 1/36
//   D3Q27: 0 -> 8/27, 1 -> 2/27, 2 -> 1/54, 3 -> 1/216
// ---------------------------------------------------------------------------
struct Lattice {
  int Q = 0;
  int c[27][3];
  double w[27];
  int opp[27];
};

Lattice make_lattice(int Q) {
  Lattice L;
  L.Q = 0;
  for (int cz = -1; cz <= 1; ++cz)
    for (int cy = -1; cy <= 1; ++cy)
      for (int cx = -1; cx <= 1; ++cx) {
        int n2 = cx * cx + cy * cy + cz * cz;
        if (Q == 19 && n2 == 3) continue;
        double w;
        if (Q == 19) w = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        else w = (n2 == 0) ? 8.0 / 27.0 : (n2 == 1 ? 2.0 / 27.0 : (n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
        L.c[L.Q][0] = cx; L.c[L.Q][1] = cy; L.c[L.Q][2] = cz;
        L.w[L.Q] = w;
        L.Q++;
      }
  for (int i = 0; i < L.Q; ++i)
    for (int j = 0; j < L.Q; ++j)
      if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] && L.c[j][2] == -L.c[i][2])
        L.opp[i] = j;
  return L;
}

// Eq. 3, read with the sign of the u^2 term that makes the zeroth moment
// equal rho (the printed "+u^2/(2c_s^2)" is a typo):
//   f^eq_i(rho,u) = w_i rho [1 + c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)]
template <class T>
T feq(const Lattice& L, int i, T rho, const T u[3]) {
  const double cs2 = 1.0 / 3.0;
  T cu = u[0] * double(L.c[i][0]) + u[1] * double(L.c[i][1]) + u[2] * double(L.c[i][2]);
  T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  T bracket = T(1.0) + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - uu / (2.0 * cs2);
  return T(L.w[i]) * rho * bracket;
}

// Eq. 5 (direct) and Eq. 6 (relaxation-time weighted) mappings eps -> B.
template <class T>
T weighting(int mode, T eps, double tau) {
  if (mode == 0) return eps;
  T t(tau - 0.5);
  return eps * t / ((T(1.0) - eps) + t);
}

// ---------------------------------------------------------------------------
// Cumulant collision on D3Q19.  The paper runs every performance case of
// Sec. 5.1 with the cumulant operator of Geier et al. (2015), which Sec. 2.2
// lists without restating it.  Its definition, restricted to the 19 moments a D3Q19
// velocity set resolves:
//   * central moments (rho-weighted) k_abc = sum_i f_i (c_ix - u_x)^a
//     (c_iy - u_y)^b (c_iz - u_z)^c for the 19 exponent triples with
//     a, b, c in {0, 1, 2}, not all three non-zero;
//   * cumulants: of order <= 3 they equal the central moments; of order 4,
//     C_220 = k_220 - (k_200 k_020 + 2 k_110^2) / rho (and its permutations);
//   * relaxation towards the cumulant equilibrium (second order rho c_s^2
//     delta_ab, higher orders 0): the off-diagonal and deviatoric diagonal
//     second-order cumulants with the shear rate omega_s = 1/tau, their trace
//     with the bulk rate omega_b, every third-order cumulant with omega_3,
//     every fourth-order one with omega_4 (rho and u are conserved);
//   * post-collision central moments from the relaxed cumulants (the same
//     order-4 relation), and the post-collision PDFs as the solution of the
//     19 x 19 linear system sum_i M_mi(u) f*_i = k*_m.
// rates = {omega_s, omega_b, omega_3, omega_4}.
// ---------------------------------------------------------------------------
constexpr int kCumE[19][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
                              {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {0, 2, 1},
                              {1, 0, 2}, {0, 1, 2}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}};

inline int cum_index(int a, int b, int c) {
  for (int m = 0; m < 19; ++m)
    if (kCumE[m][0] == a && kCumE[m][1] == b && kCumE[m][2] == c) return m;
  return -1;
}

template <class T>
T ipow(T x, int e) {
  T r(1.0);
  for (int k = 0; k < e; ++k) r = r * x;
  return r;
}

// Solve A x = b (n x n, row-major, both overwritten) by Gaussian elimination
// with partial pivoting on the values.
template <class T>
void gauss_solve(int n, T* A, T* b, T* x) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(val(A[r * n + col])) > std::fabs(val(A[piv * n + col]))) piv = r;
    if (piv != col) {
      for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
      std::swap(b[col], b[piv]);
    }
    for (int r = col + 1; r < n; ++r) {
      const T fac = A[r * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[r * n + k] -= fac * A[col * n + k];
      b[r] -= fac * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    T acc = b[r];
    for (int k = r + 1; k < n; ++k) acc -= A[r * n + k] * x[k];
    x[r] = acc / A[r * n + r];
  }
}

template <class T>
void cumulant_post(const Lattice& L, const double rates[4], const T* f, T rho, const T u[3], T* post) {
  const double ws = rates[0], wb = rates[1], w3 = rates[2], w4 = rates[3];
  const double cs2 = 1.0 / 3.0;
  T M[19 * 19], k[19];
  for (int m = 0; m < 19; ++m) {
    k[m] = T(0.0);
    for (int i = 0; i < 19; ++i) {
      M[m * 19 + i] = ipow(T(double(L.c[i][0])) - u[0], kCumE[m][0]) * ipow(T(double(L.c[i][1])) - u[1], kCumE[m][1]) *
                      ipow(T(double(L.c[i][2])) - u[2], kCumE[m][2]);
      k[m] += M[m * 19 + i] * f[i];
    }
  }
  auto K = [&](int a, int b, int c) -> T& { return k[cum_index(a, b, c)]; };
  T kp[19];
  for (int m = 0; m < 19; ++m) kp[m] = k[m];
  auto KP = [&](int a, int b, int c) -> T& { return kp[cum_index(a, b, c)]; };
  // conserved: k_000 = rho, first-order central moments 0
  KP(0, 0, 0) = rho;
  KP(1, 0, 0) = T(0.0);
  KP(0, 1, 0) = T(0.0);
  KP(0, 0, 1) = T(0.0);
  // second order
  KP(1, 1, 0) = K(1, 1, 0) * (1.0 - ws);
  KP(1, 0, 1) = K(1, 0, 1) * (1.0 - ws);
  KP(0, 1, 1) = K(0, 1, 1) * (1.0 - ws);
  const T tr = K(2, 0, 0) + K(0, 2, 0) + K(0, 0, 2);
  const T tr_eq = rho * (3.0 * cs2);
  const T tr_post = tr + (tr_eq - tr) * wb;
  KP(2, 0, 0) = tr_post / 3.0 + (K(2, 0, 0) - tr / 3.0) * (1.0 - ws);
  KP(0, 2, 0) = tr_post / 3.0 + (K(0, 2, 0) - tr / 3.0) * (1.0 - ws);
  KP(0, 0, 2) = tr_post / 3.0 + (K(0, 0, 2) - tr / 3.0) * (1.0 - ws);
  // third order: cumulant = central moment, equilibrium 0
  const int third[6][3] = {{2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}};
  for (auto& e : third) KP(e[0], e[1], e[2]) = K(e[0], e[1], e[2]) * (1.0 - w3);
  // fourth order: the three C_aab b-type cumulants of D3Q19
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};  // (x,y), (x,z), (y,z)
  for (auto& pr : pairs) {
    int e4[3] = {0, 0, 0}, ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0}, eab[3] = {0, 0, 0};
    e4[pr[0]] = 2; e4[pr[1]] = 2;
    ea[pr[0]] = 2;
    eb[pr[1]] = 2;
    eab[pr[0]] = 1; eab[pr[1]] = 1;
    const T Kab = K(eab[0], eab[1], eab[2]);
    const T C4 = K(e4[0], e4[1], e4[2]) - (K(ea[0], ea[1], ea[2]) * K(eb[0], eb[1], eb[2]) + 2.0 * Kab * Kab) / rho;
    const T C4p = C4 * (1.0 - w4);
    const T KPab = KP(eab[0], eab[1], eab[2]);
    KP(e4[0], e4[1], e4[2]) =
        C4p + (KP(ea[0], ea[1], ea[2]) * KP(eb[0], eb[1], eb[2]) + 2.0 * KPab * KPab) / rho;
  }
  gauss_solve(19, M, kp, post);
}

}  // namespace

// ---------------------------------------------------------------------------
// Plain C configuration passed from Python (ctypes).
// ---------------------------------------------------------------------------
extern "C" {

typedef struct {
  int Q;                 // 19 or 27
  int nx, ny, nz;
  int bc_z;              // 0: periodic, 1: equilibrium ghost planes at z=-1 and z=nz
  int walls_y;           // oracle-only: 1 = half-way bounce-back walls at y=-1/2, y=ny-1/2
  double wall_u_lo[3];   // velocity of the y=-1/2 wall
  double wall_u_hi[3];   // velocity of the y=ny-1/2 wall
  double force[3];       // oracle-only constant body force (Guo forcing)
  double rho0;           // reference density (ghost planes hold f^eq(rho0, u_in))
  double u_in[3];        // inflow velocity held by the ghost planes
  int fluid;             // 0: BGK (Eq. 2), 1: TRT, 2: cumulant (D3Q19)
  double tau;            // relaxation time (TRT: 1/omega_plus)
  double trt_lambda;     // TRT magic parameter Lambda
  int solid;             // 1, 2, 3: SC1 (Eq. 7), SC2 (Eq. 8), SC3 (Eq. 9)
  int weighting;         // 0: B = eps (Eq. 5); 1: tau-weighted (Eq. 6)
  double cum_rates[3];   // cumulant (fluid 2): omega_bulk, omega_3, omega_4
  int z0;                // world z index of plane 0: the lattice is the slab [z0, z0 + nz) of a larger
                         // domain (cell centres, hence the remap, u_s and the torque lever arm, use z + z0)
} or_config;

}  // extern "C"

namespace {

// A rigid body: binary super-sampled geometry field (Sec. 3) in its own frame,
// plus its rigid motion.  The geometry field holds one byte per sub-cell
// (1 = sub-cell centre inside the body) over nsx*nsy*nsz sub-cells of size
// h = 2^-s covering the body-frame box [lo, lo + (nsx, nsy, nsz) h).
template <class T>
struct Body {
  std::vector<uint8_t> sub;
  int nsx = 0, nsy = 0, nsz = 0, s = 0;
  double lo[3] = {0, 0, 0};
  double Q0[9];          // initial orientation, world <- body, row-major
  double R0[3];          // reference point (centre of rotation / mass) at step 0
  T omega[3];            // angular velocity (rad / step), world frame: u_s
  double omega_pose[3];  // angular velocity that moves the geometry (pose)
  double v[3];           // translation velocity (cells / step)
  // Two-way coupling (or_set_body_dynamics; value type only): the body moves
  // under the force and torque the fluid exerts on it at each step.
  bool free_body = false;
  double mass = 0.0, Ib[9], Ibinv[9], Fext[3], Text[3];  // body-frame inertia, external loads (world)
  double Rd[3], vd[3], Qd[9], wd[3], Ld[3];              // state: position, velocity, orientation, omega, L
};

// omega = Q Ib^-1 Q^T L (world frame)
void omega_from_L(const double Q[9], const double Ibinv[9], const double L[3], double w[3]) {
  double a[3], b[3];
  for (int i = 0; i < 3; ++i) a[i] = Q[0 * 3 + i] * L[0] + Q[1 * 3 + i] * L[1] + Q[2 * 3 + i] * L[2];  // Q^T L
  for (int i = 0; i < 3; ++i) b[i] = Ibinv[3 * i + 0] * a[0] + Ibinv[3 * i + 1] * a[1] + Ibinv[3 * i + 2] * a[2];
  for (int i = 0; i < 3; ++i) w[i] = Q[3 * i + 0] * b[0] + Q[3 * i + 1] * b[1] + Q[3 * i + 2] * b[2];
}

// Q <- Rot(phi) Q, the rotation by the angle |phi| about phi / |phi| (Rodrigues)
void rotate_by(double Q[9], const double phi[3]) {
  const double a = std::sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  if (!(a > 0.0)) return;
  const double k[3] = {phi[0] / a, phi[1] / a, phi[2] / a};
  const double c = std::cos(a), s = std::sin(a), oc = 1.0 - c;
  const double Rm[9] = {c + oc * k[0] * k[0],        oc * k[0] * k[1] - s * k[2], oc * k[0] * k[2] + s * k[1],
                        oc * k[1] * k[0] + s * k[2], c + oc * k[1] * k[1],        oc * k[1] * k[2] - s * k[0],
                        oc * k[2] * k[0] - s * k[1], oc * k[2] * k[1] + s * k[0], c + oc * k[2] * k[2]};
  double out[9];
  for (int r = 0; r < 3; ++r)
    for (int col = 0; col < 3; ++col)
      out[3 * r + col] = Rm[3 * r + 0] * Q[col] + Rm[3 * r + 1] * Q[3 + col] + Rm[3 * r + 2] * Q[6 + col];
  for (int k2 = 0; k2 < 9; ++k2) Q[k2] = out[k2];
}

// Pose of a body at step n (Sec. 3: the cell centre is multiplied by a rotation
// matrix and shifted by a translation).  Rotation about the axis omega/|omega|
// by the angle |omega| n (Rodrigues' formula), applied after Q0:
//   Q_n = [cos(th) I + sin(th) [k]_x + (1 - cos(th)) k k^T] Q0,  th = |omega| n
//   R_n = R0 + v n
// The pose uses its own copy of omega (omega_pose): the geometry sequence
// stays frozen when u_s's omega is perturbed (finite differences) or
// differentiated (tangent-linear model), since eps is piecewise constant in
// omega.
struct Pose {
  double Q[9];
  double R[3];
};

Pose pose_at(const double Q0[9], const double R0[3], const double om[3], const double v[3], long n) {
  Pose P;
  double wn = std::sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
  double Rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (wn > 0.0) {
    double k[3] = {om[0] / wn, om[1] / wn, om[2] / wn};
    double th = wn * double(n);
    double c = std::cos(th), s = std::sin(th), oc = 1.0 - c;
    Rot[0] = c + oc * k[0] * k[0];
    Rot[1] = oc * k[0] * k[1] - s * k[2];
    Rot[2] = oc * k[0] * k[2] + s * k[1];
    Rot[3] = oc * k[1] * k[0] + s * k[2];
    Rot[4] = c + oc * k[1] * k[1];
    Rot[5] = oc * k[1] * k[2] - s * k[0];
    Rot[6] = oc * k[2] * k[0] - s * k[1];
    Rot[7] = oc * k[2] * k[1] + s * k[0];
    Rot[8] = c + oc * k[2] * k[2];
  }
  for (int r = 0; r < 3; ++r)
    for (int col = 0; col < 3; ++col)
      P.Q[3 * r + col] = (Rot[3 * r + 0] * Q0[0 + col] + Rot[3 * r + 1] * Q0[3 + col]) + Rot[3 * r + 2] * Q0[6 + col];
  for (int k = 0; k < 3; ++k) P.R[k] = R0[k] + v[k] * double(n);
  return P;
}

// Sec. 3 remap for one body and one cell: transform the cell centre into the
// body frame, X = Q_n^T (x_c - R_n), take the cube of 2^s x 2^s x 2^s sub-cells
// whose lower corner is the sub-grid point nearest to X - 1/2, and average its
// bits (bits outside the stored box are 0).  In sub-cell units of the stored
// box the corner sits at ((X - 1/2) - lo) 2^s, so the first sub-cell index per
// axis is a0 = floor(((X - 1/2) - lo) 2^s + 1/2), evaluated in double in
// exactly that order (no contraction).
double remap_cell(const uint8_t* sub, int nsx, int nsy, int nsz, int s, const double lo[3],
                  const Pose& P, int x, int y, int z) {
  const int n = 1 << s;
  const double xc[3] = {double(x) + 0.5, double(y) + 0.5, double(z) + 0.5};
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = xc[k] - P.R[k];
  long a0[3];
  for (int k = 0; k < 3; ++k) {
    // column k of Q (world <- body) is row k of Q^T
    const double X = (P.Q[0 * 3 + k] * d[0] + P.Q[1 * 3 + k] * d[1]) + P.Q[2 * 3 + k] * d[2];
    a0[k] = (long)std::floor(((X - 0.5) - lo[k]) * double(n) + 0.5);
  }
  long count = 0;
  for (long az = a0[2]; az < a0[2] + n; ++az)
    for (long ay = a0[1]; ay < a0[1] + n; ++ay)
      for (long ax = a0[0]; ax < a0[0] + n; ++ax) {
        if (ax < 0 || ay < 0 || az < 0 || ax >= nsx || ay >= nsy || az >= nsz) continue;
        count += sub[((long)az * nsy + ay) * nsx + ax];
      }
  return double(count) / double(n * n * n);
}

template <class T>
struct Sim {
  or_config cfg;
  Lattice L;
  long ncell = 0;
  std::vector<T> f, post;     // f[i*ncell + cell]
  std::vector<T> delta;       // per-cell additive perturbation of eps (may be empty)
  std::vector<Body<T>> bodies;
  std::vector<T> ft;          // per step, per body: F_body[3], T_body[3] (= -S_F, -S_T)
  T u_in[3];
  long step = 0;
  int nthreads = 1;

  long cell(int x, int y, int z) const { return ((long)z * cfg.ny + y) * cfg.nx + x; }

  // The state arrays are allocated on first use, so that a simulation used
  // only for one-cell collisions (collide_at) of a huge grid stays small.
  void ensure_state() {
    if (f.empty()) {
      f.assign((size_t)L.Q * ncell, T(0.0));
      post.assign((size_t)L.Q * ncell, T(0.0));
    }
  }

  // Ghost-plane populations: f^eq_i(rho0, u_in) (reading of the unstated
  // inflow/outflow condition: equilibrium planes at z=-1 and z=nz).
  T ghost(int i) const { return feq<T>(L, i, T(cfg.rho0), u_in); }

  // Is the upstream cell x - c_i of (x,y,z) outside the domain in z?
  bool inflow_from_ghost(int i, int z) const {
    if (cfg.bc_z == 0) return false;
    int zs = z - L.c[i][2];
    return zs < 0 || zs >= cfg.nz;
  }

  void init_eq(T rho, const T u[3]) {
    ensure_state();
    for (int i = 0; i < L.Q; ++i)
      for (int z = 0; z < cfg.nz; ++z)
        for (int y = 0; y < cfg.ny; ++y)
          for (int x = 0; x < cfg.nx; ++x) {
            // The ghost planes hold their state from t = 0 on: populations that
            // enter the domain from a ghost plane take the ghost value.
            f[i * ncell + cell(x, y, z)] = inflow_from_ghost(i, z) ? ghost(i) : feq<T>(L, i, rho, u);
          }
  }

  // eps and owner body of every cell at the pose of step n (Sec. 3).  With
  // several bodies: eps = min(1, sum_b eps_b), owner = argmax_b eps_b (lower
  // id on ties), -1 where eps = 0.
  void remap_all(long n, std::vector<double>& eps, std::vector<int>& owner) const {
    eps.assign(ncell, 0.0);
    owner.assign(ncell, -1);
    std::vector<double> best(ncell, 0.0);
    const std::vector<Pose> poses = poses_at(n);
    for (size_t b = 0; b < bodies.size(); ++b) {
      const Body<T>& B = bodies[b];
      const Pose& P = poses[b];
      for (int z = 0; z < cfg.nz; ++z)
        for (int y = 0; y < cfg.ny; ++y)
          for (int x = 0; x < cfg.nx; ++x) {
            double e = remap_cell(B.sub.data(), B.nsx, B.nsy, B.nsz, B.s, B.lo, P, x, y, z + cfg.z0);
            long c = cell(x, y, z);
            eps[c] += e;
            if (e > best[c]) { best[c] = e; owner[c] = (int)b; }
          }
    }
    for (long c = 0; c < ncell; ++c) eps[c] = std::min(1.0, eps[c]);
  }

  // TRT rates: omega+ = 1/tau, Lambda = (1/omega+ - 1/2)(1/omega- - 1/2).
  double omega_plus() const { return 1.0 / cfg.tau; }
  double omega_minus() const { return 1.0 / (cfg.trt_lambda / (cfg.tau - 0.5) + 0.5); }

  std::vector<Pose> poses_at(long n) const {
    std::vector<Pose> poses;
    for (auto& B : bodies) {
      if (B.free_body) {
        Pose P;
        for (int k = 0; k < 9; ++k) P.Q[k] = B.Qd[k];
        for (int k = 0; k < 3; ++k) P.R[k] = B.Rd[k];
        poses.push_back(P);
      } else {
        poses.push_back(pose_at(B.Q0, B.R0, B.omega_pose, B.v, n));
      }
    }
    return poses;
  }

  // Two-way coupling, one explicit step of the rigid-body equations of motion
  // (semi-implicit Euler, dt = 1) with the force F and torque Tq on the body of
  // this step (about R_n):
  //   v += (F + Fext) / m,  R += v,  L += Tq + Text,
  //   Q <- Rot(w*) Q with w* = Q Ib^-1 Q^T L,  then w = Q Ib^-1 Q^T L;
  // the next step's remap, u_s and lever arm use (R, Q, v, w).
  void integrate_free(Body<T>& B, const double F[3], const double Tq[3]) {
    for (int k = 0; k < 3; ++k) B.vd[k] += (F[k] + B.Fext[k]) / B.mass;
    for (int k = 0; k < 3; ++k) B.Rd[k] += B.vd[k];
    for (int k = 0; k < 3; ++k) B.Ld[k] += Tq[k] + B.Text[k];
    double ws[3];
    omega_from_L(B.Qd, B.Ibinv, B.Ld, ws);
    rotate_by(B.Qd, ws);
    omega_from_L(B.Qd, B.Ibinv, B.Ld, B.wd);
    for (int k = 0; k < 3; ++k) {
      B.omega[k] = T(B.wd[k]);
      B.v[k] = B.vd[k];
    }
  }

  // eps and owner of one cell at the pose of step n (same rule as remap_all)
  void remap_one(const std::vector<Pose>& poses, int x, int y, int z, double& eps_c, int& owner_c) const {
    double sum = 0.0, best = 0.0;
    owner_c = -1;
    for (size_t b = 0; b < bodies.size(); ++b) {
      const Body<T>& B = bodies[b];
      double e = remap_cell(B.sub.data(), B.nsx, B.nsy, B.nsz, B.s, B.lo, poses[b], x, y, z + cfg.z0);
      sum += e;
      if (e > best) { best = e; owner_c = (int)b; }
    }
    eps_c = std::min(1.0, sum);
  }

  // One cell's collision (Eq. 4 with Eq. 2 / TRT, Eq. 5 / 6, Eq. 7 / 8 / 9) from
  // the pre-collision state f: post-collision PDFs post[Q] and the cell's
  // force density g = B sum_i Omega^S_i c_i.
  void collide_cell(int x, int y, int z, double eps_c, int owner_c, const std::vector<Pose>& poses, T* post,
                    T* g) const {
    const long c = cell(x, y, z);
    T fl[27];
    for (int i = 0; i < L.Q; ++i) fl[i] = f[i * ncell + c];
    collide_given(x, y, z, eps_c, owner_c, poses, fl, post, g);
  }

  // The same collision from explicitly given pre-collision PDFs fl[Q] of cell
  // (x, y, z) (the per-cell delta still applies).
  void collide_given(int x, int y, int z, double eps_c, int owner_c, const std::vector<Pose>& poses, const T* fl,
                     T* post, T* g) const {
    const int Q = L.Q;
    const double tau = cfg.tau;
    const double cs2 = 1.0 / 3.0;
    const double om_p = omega_plus(), om_m = omega_minus();
    const long c = cell(x, y, z);
    T E[27], G[27], OF[27], OS[27];
    // moments of the pre-collision PDFs
    T rho(0.0), j[3] = {T(0.0), T(0.0), T(0.0)};
    for (int i = 0; i < Q; ++i) {
      rho += fl[i];
      for (int k = 0; k < 3; ++k) j[k] += fl[i] * double(L.c[i][k]);
    }
    T u[3];
    T Fb[3] = {T(cfg.force[0]), T(cfg.force[1]), T(cfg.force[2])};
    // Guo forcing (oracle-only, for the Poiseuille pin): u = (j + F/2)/rho
    for (int k = 0; k < 3; ++k) u[k] = (j[k] + Fb[k] * 0.5) / rho;
    // solid fraction and weighting, Eq. 5 / Eq. 6
    T e(eps_c);
    if (!delta.empty()) e = e + delta[c];
    T Bw = weighting<T>(cfg.weighting, e, tau);
    // solid velocity u_s = omega x (x_c - R_n) + v of the owner body
    T us[3] = {T(0.0), T(0.0), T(0.0)};
    if (owner_c >= 0) {
      const Body<T>& Bd = bodies[owner_c];
      T r[3] = {T(x + 0.5 - poses[owner_c].R[0]), T(y + 0.5 - poses[owner_c].R[1]),
                T((z + cfg.z0) + 0.5 - poses[owner_c].R[2])};
      us[0] = Bd.omega[1] * r[2] - Bd.omega[2] * r[1] + Bd.v[0];
      us[1] = Bd.omega[2] * r[0] - Bd.omega[0] * r[2] + Bd.v[1];
      us[2] = Bd.omega[0] * r[1] - Bd.omega[1] * r[0] + Bd.v[2];
    }
    for (int i = 0; i < Q; ++i) {
      E[i] = feq<T>(L, i, rho, u);    // f^eq(rho, u)
      G[i] = feq<T>(L, i, rho, us);   // f^eq(rho, u_s)
    }
    // fluid collision: Eq. 2 (BGK), two-relaxation-time, or cumulant
    if (cfg.fluid == 2) {
      const double rates[4] = {1.0 / tau, cfg.cum_rates[0], cfg.cum_rates[1], cfg.cum_rates[2]};
      T cp[27];
      cumulant_post<T>(L, rates, fl, rho, u, cp);
      for (int i = 0; i < Q; ++i) OF[i] = cp[i] - fl[i];
    }
    for (int i = 0; i < Q && cfg.fluid != 2; ++i) {
      const int ib = L.opp[i];
      if (cfg.fluid == 0) {
        OF[i] = -(fl[i] - E[i]) / tau;
      } else {
        T fp = (fl[i] + fl[ib]) * 0.5, fm = (fl[i] - fl[ib]) * 0.5;
        T ep = (E[i] + E[ib]) * 0.5, em = (E[i] - E[ib]) * 0.5;
        OF[i] = -(fp - ep) * om_p - (fm - em) * om_m;
      }
    }
    // solid collision, Eq. 7 (SC1), Eq. 8 (SC2, as printed: u_s in both
    // brackets), Eq. 9 (SC3)
    for (int i = 0; i < Q; ++i) {
      const int ib = L.opp[i];
      if (cfg.solid == 1) {
        OS[i] = (fl[ib] - E[ib]) - (fl[i] - G[i]);
      } else if (cfg.solid == 2) {
        OS[i] = (G[i] - fl[i]) + (fl[i] - G[i]) * (1.0 - 1.0 / tau);
      } else {
        OS[i] = (fl[ib] - G[ib]) - (fl[i] - G[i]);
      }
    }
    // PSM rule, Eq. 4
    T gs[3] = {T(0.0), T(0.0), T(0.0)};
    for (int i = 0; i < Q; ++i) {
      T one_minus_B = T(1.0) - Bw;
      post[i] = fl[i] + one_minus_B * OF[i] + Bw * OS[i];
      for (int k = 0; k < 3; ++k) gs[k] += OS[i] * double(L.c[i][k]);
    }
    for (int k = 0; k < 3; ++k) g[k] = Bw * gs[k];
    // Guo forcing source (oracle-only)
    if (cfg.force[0] != 0.0 || cfg.force[1] != 0.0 || cfg.force[2] != 0.0) {
      T S[27];
      for (int i = 0; i < Q; ++i) {
        T cu = u[0] * double(L.c[i][0]) + u[1] * double(L.c[i][1]) + u[2] * double(L.c[i][2]);
        T acc(0.0);
        for (int k = 0; k < 3; ++k)
          acc += ((double(L.c[i][k]) - u[k]) / cs2 + cu * double(L.c[i][k]) / (cs2 * cs2)) * Fb[k];
        S[i] = T(L.w[i]) * acc;
      }
      for (int i = 0; i < Q; ++i) {
        const int ib = L.opp[i];
        if (cfg.fluid == 0) {
          post[i] += S[i] * (1.0 - 0.5 / tau);
        } else {
          T sp = (S[i] + S[ib]) * 0.5, sm = (S[i] - S[ib]) * 0.5;
          post[i] += sp * (1.0 - 0.5 * om_p) + sm * (1.0 - 0.5 * om_m);
        }
      }
    }
  }

  // f_i(x, n + 1) for sampled cells x, computed one by one from the current
  // state f at step n: the collision of every upstream cell x - c_i, then the
  // streaming rule of Eq. 1 (periodic x / y, ghost planes or periodic z).  No
  // half-way walls or body force here.  out[k * Q + i].
  void update_cells(const long* cells, long ncells_req, T* out) const {
    const std::vector<Pose> poses = poses_at(step);
    const int Q = L.Q;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (long k = 0; k < ncells_req; ++k) {
      const long c = cells[k];
      const int x = (int)(c % cfg.nx), y = (int)((c / cfg.nx) % cfg.ny), z = (int)(c / ((long)cfg.nx * cfg.ny));
      T post[27], g[3];
      for (int i = 0; i < Q; ++i) {
        int xs = ((x - L.c[i][0]) % cfg.nx + cfg.nx) % cfg.nx;
        int ys = ((y - L.c[i][1]) % cfg.ny + cfg.ny) % cfg.ny;
        int zs = z - L.c[i][2];
        if (zs < 0 || zs >= cfg.nz) {
          if (cfg.bc_z == 1) { out[k * Q + i] = ghost(i); continue; }
          zs = (zs + cfg.nz) % cfg.nz;
        }
        double e;
        int o;
        remap_one(poses, xs, ys, zs, e, o);
        collide_cell(xs, ys, zs, e, o, poses, post, g);
        out[k * Q + i] = post[i];
      }
    }
  }

  void do_step() {
    ensure_state();
    const int Q = L.Q;
    const int nx = cfg.nx, ny = cfg.ny, nz = cfg.nz;
    const double tau = cfg.tau;
    std::vector<double> eps;
    std::vector<int> owner;
    remap_all(step, eps, owner);
    const std::vector<Pose> poses = poses_at(step);
    const int nb = (int)bodies.size();
    // Per-cell force density g = B sum_i Omega^S_i c_i, kept for the
    // force/torque sums below (computed in a fixed order afterwards).
    std::vector<T> g(3 * ncell, T(0.0));

#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int z = 0; z < nz; ++z) {
      T pc[27];
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const long c = cell(x, y, z);
          collide_cell(x, y, z, eps[c], owner[c], poses, pc, &g[3 * c]);
          for (int i = 0; i < Q; ++i) post[i * ncell + c] = pc[i];
        }
    }

    // Force and torque, Eq. 10 and Eq. 11 (dx = dt = 1), summed over the cells
    // in contact (B > 0) of each body in the fixed order z, y, x.  The paper's
    // sums S are the momentum the solid gives the fluid; the force and torque
    // ON THE BODY are their negatives, which is what is recorded.
    for (int b = 0; b < nb; ++b) {
      T SF[3] = {T(0.0), T(0.0), T(0.0)}, ST[3] = {T(0.0), T(0.0), T(0.0)};
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const long c = cell(x, y, z);
            if (owner[c] != b) continue;
            T e(eps[c]);
            if (!delta.empty()) e = e + delta[c];
            T Bw = weighting<T>(cfg.weighting, e, tau);
            if (!(val(Bw) > 0.0)) continue;
            T r[3] = {T(x + 0.5 - poses[b].R[0]), T(y + 0.5 - poses[b].R[1]),
                      T((z + cfg.z0) + 0.5 - poses[b].R[2])};
            const T* gc = &g[3 * c];
            for (int k = 0; k < 3; ++k) SF[k] += gc[k];
            ST[0] += r[1] * gc[2] - r[2] * gc[1];
            ST[1] += r[2] * gc[0] - r[0] * gc[2];
            ST[2] += r[0] * gc[1] - r[1] * gc[0];
          }
      for (int k = 0; k < 3; ++k) ft.push_back(-SF[k]);
      for (int k = 0; k < 3; ++k) ft.push_back(-ST[k]);
    }
    for (int b = 0; b < nb; ++b) {
      if (!bodies[b].free_body) continue;
      const size_t o = ft.size() - (size_t)(nb - b) * 6;
      const double F[3] = {val(ft[o]), val(ft[o + 1]), val(ft[o + 2])};
      const double Tq[3] = {val(ft[o + 3]), val(ft[o + 4]), val(ft[o + 5])};
      integrate_free(bodies[b], F, Tq);
    }

    // Streaming, Eq. 1: f_i(x + c_i, t + 1) = post_i(x), read as a pull from
    // x - c_i.  Periodic in x and y (and z when bc_z = 0); from the ghost plane
    // when x - c_i lies outside in z; half-way bounce-back (oracle-only) when
    // x - c_i lies beyond a y wall.
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const long c = cell(x, y, z);
          for (int i = 0; i < Q; ++i) {
            int xs = x - L.c[i][0], ys = y - L.c[i][1], zs = z - L.c[i][2];
            xs = (xs + nx) % nx;
            if (cfg.walls_y) {
              if (ys < 0 || ys >= ny) {
                const double* uw = (ys < 0) ? cfg.wall_u_lo : cfg.wall_u_hi;
                double cuw = L.c[i][0] * uw[0] + L.c[i][1] * uw[1] + L.c[i][2] * uw[2];
                f[i * ncell + c] = post[L.opp[i] * ncell + c] + T(6.0 * L.w[i] * cfg.rho0 * cuw);
                continue;
              }
            } else {
              ys = (ys + ny) % ny;
            }
            if (zs < 0 || zs >= nz) {
              if (cfg.bc_z == 1) { f[i * ncell + c] = ghost(i); continue; }
              zs = (zs + nz) % nz;
            }
            f[i * ncell + c] = post[i * ncell + cell(xs, ys, zs)];
          }
        }
    step++;
  }
};

template <class T>
Sim<T>* make_sim(const or_config* cfg) {
  if (cfg->Q != 19 && cfg->Q != 27) return nullptr;
  if (cfg->nx <= 0 || cfg->ny <= 0 || cfg->nz <= 0) return nullptr;
  // the cumulant operator is defined here on D3Q19 only, without a body force
  if (cfg->fluid == 2 && (cfg->Q != 19 || cfg->force[0] != 0.0 || cfg->force[1] != 0.0 || cfg->force[2] != 0.0))
    return nullptr;
  auto* S = new Sim<T>();
  S->cfg = *cfg;
  S->L = make_lattice(cfg->Q);
  S->ncell = (long)cfg->nx * cfg->ny * cfg->nz;
  for (int k = 0; k < 3; ++k) S->u_in[k] = T(cfg->u_in[k]);
#ifdef _OPENMP
  S->nthreads = omp_get_max_threads();
#endif
  return S;
}

template <class T>
int add_body(Sim<T>* S, const uint8_t* sub, int nsx, int nsy, int nsz, int s, const double lo[3],
             const double Q0[9], const double R0[3], const double omega[3], const double v[3]) {
  Body<T> B;
  B.sub.assign(sub, sub + (size_t)nsx * nsy * nsz);
  B.nsx = nsx; B.nsy = nsy; B.nsz = nsz; B.s = s;
  for (int k = 0; k < 3; ++k) {
    B.lo[k] = lo[k]; B.R0[k] = R0[k]; B.omega[k] = T(omega[k]); B.omega_pose[k] = omega[k]; B.v[k] = v[k];
  }
  for (int k = 0; k < 9; ++k) B.Q0[k] = Q0[k];
  S->bodies.push_back(B);
  return (int)S->bodies.size() - 1;
}

// ---------------------------------------------------------------------------
// Analytic bodies, voxelised onto the sub-cell grid (bit = sub-cell centre
// inside).  Box rule: per axis, lo = -(floor(half extent) + 2), and
// 2 (floor(half extent) + 2) coarse cells, so the sub-grid lines fall on
// integers of the body frame.
// ---------------------------------------------------------------------------
struct RotorSpec {
  double r_hub, hub_len, span, chord, thickness, pitch_root_deg, twist_deg, phase;
  int n_blades, hand;
};

bool inside_shape(int kind, const double* p, double x, double y, double z) {
  if (kind == 0) {  // sphere radius p[0]
    return x * x + y * y + z * z <= p[0] * p[0];
  } else if (kind == 1) {  // ellipsoid semi-axes p[0..2]
    double a = x / p[0], b = y / p[1], c = z / p[2];
    return a * a + b * b + c * c <= 1.0;
  } else if (kind == 2) {  // box half-extents p[0..2]
    return std::fabs(x) <= p[0] && std::fabs(y) <= p[1] && std::fabs(z) <= p[2];
  }
  // rotor: hub cylinder plus twisted thin elliptic blades
  RotorSpec R;
  R.r_hub = p[0]; R.hub_len = p[1]; R.span = p[2]; R.chord = p[3]; R.thickness = p[4];
  R.pitch_root_deg = p[5]; R.twist_deg = p[6]; R.phase = p[7];
  R.n_blades = (int)p[8]; R.hand = (int)p[9];
  const double PI = 3.14159265358979323846;
  double r = std::sqrt(x * x + y * y);
  if (r <= R.r_hub && std::fabs(z) <= 0.5 * R.hub_len) return true;
  if (r < R.r_hub || r > R.r_hub + R.span) return false;
  double phi = std::atan2(y, x);
  double beta = (R.pitch_root_deg - R.twist_deg * (r - R.r_hub) / R.span) * (PI / 180.0) * double(R.hand);
  double cb = std::cos(beta), sb = std::sin(beta);
  double ha = 0.5 * R.chord, hb = 0.5 * R.thickness;
  for (int k = 0; k < R.n_blades; ++k) {
    double dphi = phi - (R.phase + 2.0 * PI * double(k) / double(R.n_blades));
    dphi = dphi - 2.0 * PI * std::floor((dphi + PI) / (2.0 * PI));
    double t = r * dphi;
    double xi = t * cb + z * sb;
    double eta = -t * sb + z * cb;
    double qa = xi / ha, qb = eta / hb;
    if (qa * qa + qb * qb <= 1.0) return true;
  }
  return false;
}

void shape_half_extent(int kind, const double* p, double he[3]) {
  if (kind == 0) { he[0] = he[1] = he[2] = p[0]; }
  else if (kind == 1 || kind == 2) { he[0] = p[0]; he[1] = p[1]; he[2] = p[2]; }
  else {
    double rt = p[0] + p[2];
    double ax = 0.5 * std::sqrt(p[3] * p[3] + p[4] * p[4]);
    he[0] = he[1] = rt;
    he[2] = std::max(0.5 * p[1], ax);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (ctypes).  "or_" = double, "ort_" = tangent-linear (Dual).
// ---------------------------------------------------------------------------
extern "C" {

int or_lattice(int Q, int* c, double* w, int* opp) {
  if (Q != 19 && Q != 27) return -1;
  Lattice L = make_lattice(Q);
  for (int i = 0; i < Q; ++i) {
    for (int k = 0; k < 3; ++k) c[3 * i + k] = L.c[i][k];
    w[i] = L.w[i];
    opp[i] = L.opp[i];
  }
  return 0;
}

double or_feq(int Q, int i, double rho, const double* u) {
  Lattice L = make_lattice(Q);
  return feq<double>(L, i, rho, u);
}

double or_weighting(int mode, double eps, double tau) { return weighting<double>(mode, eps, tau); }

// Body box rule and voxelisation of an analytic shape.
//   kind: 0 sphere(r), 1 ellipsoid(a,b,c), 2 box(hx,hy,hz),
//         3 rotor(r_hub, hub_len, span, chord, thickness, pitch_root_deg,
//                 twist_deg, phase_rad, n_blades, hand)
// dims_out[3] = coarse cells per axis, lo_out[3] = body-frame box origin.
int or_shape_box(int kind, const double* p, int* dims_out, double* lo_out) {
  double he[3];
  shape_half_extent(kind, p, he);
  for (int k = 0; k < 3; ++k) {
    int m = (int)std::floor(he[k]) + 2;
    dims_out[k] = 2 * m;
    lo_out[k] = -(double)m;
  }
  return 0;
}

// sub_out: (dims*2^s) sub-cells, z-major, x fastest; 1 = centre inside.
int or_voxelize(int kind, const double* p, int s, uint8_t* sub_out) {
  int dims[3];
  double lo[3];
  or_shape_box(kind, p, dims, lo);
  const int n = 1 << s;
  const double h = 1.0 / double(n);
  const long nsx = (long)dims[0] * n, nsy = (long)dims[1] * n, nsz = (long)dims[2] * n;
#pragma omp parallel for schedule(static)
  for (long az = 0; az < nsz; ++az)
    for (long ay = 0; ay < nsy; ++ay)
      for (long ax = 0; ax < nsx; ++ax) {
        double x = lo[0] + (double(ax) + 0.5) * h;
        double y = lo[1] + (double(ay) + 0.5) * h;
        double z = lo[2] + (double(az) + 0.5) * h;
        sub_out[(az * nsy + ay) * nsx + ax] = inside_shape(kind, p, x, y, z) ? 1 : 0;
      }
  return 0;
}

int or_inside(int kind, const double* p, double x, double y, double z) { return inside_shape(kind, p, x, y, z) ? 1 : 0; }

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Voxelisation of a closed triangle mesh (Sec. 3: the body's surface mesh is
// turned into the super-sampled binary field once).  A sub-cell is inside iff
// a ray from its centre in the +x direction crosses the surface an odd number
// of times.  Everything is decided in exact integer arithmetic:
//   * the box of the field is [lo, lo + dims) with lo = floor(min v) - 1 and
//     lo + dims = ceil(max v) + 1 per axis (whole cells);
//   * coordinates relative to lo are quantised to integers in units of
//     2^-(s+8) cells (round half away from zero); the centre of sub-cell a is
//     256 a + 128 in those units;
//   * the ray hits the triangle's projection onto the (y, z) plane when the
//     three edge orientations have one strict sign, ties broken as if the
//     centre were moved by (delta^2, delta) in (y, z) for an infinitesimal
//     delta > 0 (simulation of simplicity: a point on a shared edge or vertex
//     belongs to exactly one side);
//   * the crossing counts when it lies at or ahead of the centre in x.
// Brute force: every sub-cell against every triangle.
// ---------------------------------------------------------------------------
struct MeshQ {
  std::vector<int64_t> v;  // quantised vertices [nv][3]
  int64_t dims[3];
  double lo[3];
};

bool mesh_box(const float* vert, long nv, int s, int64_t dims[3], double lo[3]) {
  if (nv < 3) return false;
  for (int k = 0; k < 3; ++k) {
    double mn = 1e300, mx = -1e300;
    for (long i = 0; i < nv; ++i) {
      const double c = (double)vert[3 * i + k];
      if (!std::isfinite(c)) return false;
      mn = std::min(mn, c);
      mx = std::max(mx, c);
    }
    lo[k] = std::floor(mn) - 1.0;
    dims[k] = (int64_t)(std::ceil(mx) + 1.0 - lo[k]);
    if (dims[k] < 1 || dims[k] > ((int64_t)1 << (19 - s))) return false;
  }
  return true;
}

// sign of the (y, z) orientation of P against the directed edge a -> b, with
// the symbolic perturbation of P by (delta^2, delta)
int orient_yz(const int64_t* a, const int64_t* b, int64_t py, int64_t pz) {
  const int64_t ey = b[1] - a[1], ez = b[2] - a[2];
  const int64_t o = ey * (pz - a[2]) - ez * (py - a[1]);
  if (o != 0) return o > 0 ? 1 : -1;
  if (ey != 0) return ey > 0 ? 1 : -1;
  if (ez != 0) return ez < 0 ? 1 : -1;
  return 0;
}

// does the +x ray from P cross triangle (a, b, c) at or ahead of P?
bool ray_crosses(const int64_t* a, const int64_t* b, const int64_t* c, int64_t px, int64_t py, int64_t pz) {
  const int s1 = orient_yz(a, b, py, pz), s2 = orient_yz(b, c, py, pz), s3 = orient_yz(c, a, py, pz);
  if (s1 == 0 || s1 != s2 || s2 != s3) return false;
  const int64_t e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const int64_t e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const int64_t nx = e1[1] * e2[2] - e1[2] * e2[1];
  const int64_t ny = e1[2] * e2[0] - e1[0] * e2[2];
  const int64_t nz = e1[0] * e2[1] - e1[1] * e2[0];
  // the ray point P + t e_x lies on the plane for t = n . (a - P) / nx
  const __int128 d = (__int128)nx * (a[0] - px) + (__int128)ny * (a[1] - py) + (__int128)nz * (a[2] - pz);
  return nx > 0 ? d >= 0 : d <= 0;
}

}  // namespace

extern "C" {

int or_mesh_box(const float* vert, long nv, int s, long* dims_out, double* lo_out) {
  int64_t dims[3];
  double lo[3];
  if (s < 0 || s > 3 || !mesh_box(vert, nv, s, dims, lo)) return -1;
  for (int k = 0; k < 3; ++k) {
    dims_out[k] = (long)dims[k];
    lo_out[k] = lo[k];
  }
  return 0;
}

// sub_out[(az * nsy + ay) * nsx + ax], n = 2^s sub-cells per cell and axis
int or_voxelize_mesh(const float* vert, long nv, const int* tri, long nt, int s, uint8_t* sub_out) {
  int64_t dims[3];
  double lo[3];
  if (s < 0 || s > 3 || !mesh_box(vert, nv, s, dims, lo)) return -1;
  const double scale = std::ldexp(1.0, s + 8);
  std::vector<int64_t> q((size_t)nv * 3);
  for (long i = 0; i < nv; ++i)
    for (int k = 0; k < 3; ++k) q[3 * i + k] = (int64_t)std::llround(((double)vert[3 * i + k] - lo[k]) * scale);
  for (long t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k)
      if (tri[3 * t + k] < 0 || tri[3 * t + k] >= nv) return -1;
  const int n = 1 << s;
  const long nsx = (long)dims[0] * n, nsy = (long)dims[1] * n, nsz = (long)dims[2] * n;
#pragma omp parallel for schedule(dynamic)
  for (long az = 0; az < nsz; ++az)
    for (long ay = 0; ay < nsy; ++ay)
      for (long ax = 0; ax < nsx; ++ax) {
        const int64_t px = 256 * (int64_t)ax + 128, py = 256 * (int64_t)ay + 128, pz = 256 * (int64_t)az + 128;
        int parity = 0;
        for (long t = 0; t < nt; ++t) {
          const int64_t* a = &q[3 * (size_t)tri[3 * t]];
          const int64_t* b = &q[3 * (size_t)tri[3 * t + 1]];
          const int64_t* c = &q[3 * (size_t)tri[3 * t + 2]];
          if (ray_crosses(a, b, c, px, py, pz)) parity ^= 1;
        }
        sub_out[(az * nsy + ay) * nsx + ax] = (uint8_t)parity;
      }
  return 0;
}


// Stand-alone remap of one body (Sec. 3) at the pose of step n over an
// nx*ny*nz grid -> eps (double, exact multiples of 2^-3s).
int or_remap(const uint8_t* sub, int nsx, int nsy, int nsz, int s, const double* lo, const double* Q0,
             const double* R0, const double* omega, const double* v, long n, int nx, int ny, int nz,
             double* eps_out) {
  Pose P = pose_at(Q0, R0, omega, v, n);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        eps_out[((long)z * ny + y) * nx + x] = remap_cell(sub, nsx, nsy, nsz, s, lo, P, x, y, z);
  return 0;
}

int or_pose(const double* Q0, const double* R0, const double* omega, const double* v, long n, double* Q_out,
            double* R_out) {
  Pose P = pose_at(Q0, R0, omega, v, n);
  for (int k = 0; k < 9; ++k) Q_out[k] = P.Q[k];
  for (int k = 0; k < 3; ++k) R_out[k] = P.R[k];
  return 0;
}

// ---------------------------- double simulation ----------------------------
void* or_create(const or_config* cfg) { return make_sim<double>(cfg); }
void or_destroy(void* h) { delete static_cast<Sim<double>*>(h); }
int or_set_threads(void* h, int n) { static_cast<Sim<double>*>(h)->nthreads = n < 1 ? 1 : n; return 0; }
int or_get_threads(void* h) { return static_cast<Sim<double>*>(h)->nthreads; }
int or_add_body(void* h, const uint8_t* sub, int nsx, int nsy, int nsz, int s, const double* lo, const double* Q0,
                const double* R0, const double* omega, const double* v) {
  return add_body(static_cast<Sim<double>*>(h), sub, nsx, nsy, nsz, s, lo, Q0, R0, omega, v);
}
// Change only the angular velocity that enters u_s (geometry stays on the
// pose of the omega given to or_add_body).
int or_set_body_us_omega(void* h, int b, const double* omega) {
  auto* S = static_cast<Sim<double>*>(h);
  if (b < 0 || b >= (int)S->bodies.size()) return -1;
  for (int k = 0; k < 3; ++k) S->bodies[b].omega[k] = omega[k];
  return 0;
}
// Two-way coupling of body b from the current step: mass, body-frame inertia
// Ib[9] (symmetric positive definite), constant external force and torque
// (world).  The state starts from the prescribed motion at the current step.
int or_set_body_dynamics(void* h, int b, double mass, const double* Ib, const double* Fext, const double* Text) {
  auto* S = static_cast<Sim<double>*>(h);
  if (b < 0 || b >= (int)S->bodies.size() || !(mass > 0.0)) return -1;
  Body<double>& B = S->bodies[b];
  const double det = Ib[0] * (Ib[4] * Ib[8] - Ib[5] * Ib[7]) - Ib[1] * (Ib[3] * Ib[8] - Ib[5] * Ib[6]) +
                     Ib[2] * (Ib[3] * Ib[7] - Ib[4] * Ib[6]);
  if (!(det > 0.0)) return -1;
  // inverse by cofactors
  B.Ibinv[0] = (Ib[4] * Ib[8] - Ib[5] * Ib[7]) / det;
  B.Ibinv[1] = (Ib[2] * Ib[7] - Ib[1] * Ib[8]) / det;
  B.Ibinv[2] = (Ib[1] * Ib[5] - Ib[2] * Ib[4]) / det;
  B.Ibinv[3] = (Ib[5] * Ib[6] - Ib[3] * Ib[8]) / det;
  B.Ibinv[4] = (Ib[0] * Ib[8] - Ib[2] * Ib[6]) / det;
  B.Ibinv[5] = (Ib[2] * Ib[3] - Ib[0] * Ib[5]) / det;
  B.Ibinv[6] = (Ib[3] * Ib[7] - Ib[4] * Ib[6]) / det;
  B.Ibinv[7] = (Ib[1] * Ib[6] - Ib[0] * Ib[7]) / det;
  B.Ibinv[8] = (Ib[0] * Ib[4] - Ib[1] * Ib[3]) / det;
  for (int k = 0; k < 9; ++k) B.Ib[k] = Ib[k];
  for (int k = 0; k < 3; ++k) {
    B.Fext[k] = Fext[k];
    B.Text[k] = Text[k];
  }
  B.mass = mass;
  const Pose P = pose_at(B.Q0, B.R0, B.omega_pose, B.v, S->step);
  for (int k = 0; k < 9; ++k) B.Qd[k] = P.Q[k];
  for (int k = 0; k < 3; ++k) {
    B.Rd[k] = P.R[k];
    B.vd[k] = B.v[k];
    B.wd[k] = B.omega[k];
  }
  // L = Q Ib Q^T w
  double a[3], c[3];
  for (int i = 0; i < 3; ++i) a[i] = B.Qd[0 * 3 + i] * B.wd[0] + B.Qd[1 * 3 + i] * B.wd[1] + B.Qd[2 * 3 + i] * B.wd[2];
  for (int i = 0; i < 3; ++i) c[i] = Ib[3 * i + 0] * a[0] + Ib[3 * i + 1] * a[1] + Ib[3 * i + 2] * a[2];
  for (int i = 0; i < 3; ++i) B.Ld[i] = B.Qd[3 * i + 0] * c[0] + B.Qd[3 * i + 1] * c[1] + B.Qd[3 * i + 2] * c[2];
  B.free_body = true;
  return 0;
}
// R[3], v[3], Q[9], omega[3], L[3] of body b (the pose of the next step to run)
int or_body_state(void* h, int b, double* out) {
  auto* S = static_cast<Sim<double>*>(h);
  if (b < 0 || b >= (int)S->bodies.size()) return -1;
  const Body<double>& B = S->bodies[b];
  if (B.free_body) {
    for (int k = 0; k < 3; ++k) out[k] = B.Rd[k], out[3 + k] = B.vd[k], out[15 + k] = B.wd[k], out[18 + k] = B.Ld[k];
    for (int k = 0; k < 9; ++k) out[6 + k] = B.Qd[k];
  } else {
    const Pose P = pose_at(B.Q0, B.R0, B.omega_pose, B.v, S->step);
    for (int k = 0; k < 3; ++k) out[k] = P.R[k], out[3 + k] = B.v[k], out[15 + k] = B.omega[k], out[18 + k] = 0.0;
    for (int k = 0; k < 9; ++k) out[6 + k] = P.Q[k];
  }
  return 0;
}
int or_init_eq(void* h, double rho, const double* u) {
  auto* S = static_cast<Sim<double>*>(h);
  S->init_eq(rho, u);
  return 0;
}
int or_set_f(void* h, const double* f) {
  auto* S = static_cast<Sim<double>*>(h);
  S->ensure_state();
  std::memcpy(S->f.data(), f, sizeof(double) * S->f.size());
  return 0;
}
int or_get_f(void* h, double* f) {
  auto* S = static_cast<Sim<double>*>(h);
  S->ensure_state();
  std::memcpy(f, S->f.data(), sizeof(double) * S->f.size());
  return 0;
}
int or_set_delta(void* h, const double* d) {
  auto* S = static_cast<Sim<double>*>(h);
  if (!d) { S->delta.clear(); return 0; }
  S->delta.assign(d, d + S->ncell);
  return 0;
}
int or_step(void* h, int n) {
  auto* S = static_cast<Sim<double>*>(h);
  for (int k = 0; k < n; ++k) S->do_step();
  return 0;
}
long or_step_count(void* h) { return static_cast<Sim<double>*>(h)->step; }
int or_ft(void* h, double* out) {  // steps * nbodies * 6, body convention
  auto* S = static_cast<Sim<double>*>(h);
  std::memcpy(out, S->ft.data(), sizeof(double) * S->ft.size());
  return (int)(S->ft.size());
}
int or_eps(void* h, long n, double* eps, int* owner) {
  auto* S = static_cast<Sim<double>*>(h);
  std::vector<double> e;
  std::vector<int> o;
  S->remap_all(n, e, o);
  std::memcpy(eps, e.data(), sizeof(double) * e.size());
  if (owner) std::memcpy(owner, o.data(), sizeof(int) * o.size());
  return 0;
}
// f_i(x, n + 1) at the listed cells from the current state (no stepping):
// out[k * Q + i] in the oracle's direction order.
int or_update_cells(void* h, const long* cells, long n, double* out) {
  auto* S = static_cast<Sim<double>*>(h);
  S->ensure_state();
  for (long k = 0; k < n; ++k)
    if (cells[k] < 0 || cells[k] >= S->ncell) return -1;
  S->update_cells(cells, n, out);
  return 0;
}
// One cell's collision at the pose of step n from given pre-collision PDFs
// f_in[Q] (oracle order): post_out[Q] and g_out[3] = B sum_i Omega^S_i c_i;
// eps and owner are computed by the remap (Sec. 3).
int or_collide_at(void* h, long n, int x, int y, int z, const double* f_in, double* post_out, double* g_out,
                  double* eps_out) {
  auto* S = static_cast<Sim<double>*>(h);
  if (x < 0 || y < 0 || z < 0 || x >= S->cfg.nx || y >= S->cfg.ny || z >= S->cfg.nz) return -1;
  const std::vector<Pose> poses = S->poses_at(n);
  double e;
  int o;
  S->remap_one(poses, x, y, z, e, o);
  double g[3];
  S->collide_given(x, y, z, e, o, poses, f_in, post_out, g);
  if (g_out) for (int k = 0; k < 3; ++k) g_out[k] = g[k];
  if (eps_out) *eps_out = e;
  return 0;
}
// rho and u = j/rho (no forcing shift) per cell
int or_macroscopic(void* h, double* rho, double* u) {
  auto* S = static_cast<Sim<double>*>(h);
  S->ensure_state();
  for (long c = 0; c < S->ncell; ++c) {
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < S->L.Q; ++i) {
      double fi = S->f[i * S->ncell + c];
      r += fi;
      for (int k = 0; k < 3; ++k) j[k] += fi * S->L.c[i][k];
    }
    rho[c] = r;
    for (int k = 0; k < 3; ++k) u[3 * c + k] = j[k] / r;
  }
  return 0;
}

// ------------------------- tangent-linear simulation ------------------------
// Seeds: d_delta (per cell, may be NULL), d_omega (per body 3, set with
// ort_add_body), d_u_in (3).  Outputs: value and tangent of every recorded
// force/torque component.
void* ort_create(const or_config* cfg, const double* d_u_in) {
  auto* S = make_sim<Dual>(cfg);
  if (!S) return nullptr;
  for (int k = 0; k < 3; ++k) S->u_in[k] = Dual(cfg->u_in[k], d_u_in ? d_u_in[k] : 0.0);
  return S;
}
void ort_destroy(void* h) { delete static_cast<Sim<Dual>*>(h); }
int ort_set_threads(void* h, int n) { static_cast<Sim<Dual>*>(h)->nthreads = n < 1 ? 1 : n; return 0; }
int ort_add_body(void* h, const uint8_t* sub, int nsx, int nsy, int nsz, int s, const double* lo, const double* Q0,
                 const double* R0, const double* omega, const double* d_omega, const double* v) {
  auto* S = static_cast<Sim<Dual>*>(h);
  int b = add_body(S, sub, nsx, nsy, nsz, s, lo, Q0, R0, omega, v);
  for (int k = 0; k < 3; ++k) S->bodies[b].omega[k] = Dual(omega[k], d_omega ? d_omega[k] : 0.0);
  return b;
}
// Equilibrium initial state at (rho, u) with tangent du (e.g. u = u_in).
int ort_init_eq(void* h, double rho, const double* u, const double* du) {
  auto* S = static_cast<Sim<Dual>*>(h);
  Dual uu[3];
  for (int k = 0; k < 3; ++k) uu[k] = Dual(u[k], du ? du[k] : 0.0);
  S->init_eq(Dual(rho), uu);
  return 0;
}
int ort_set_delta(void* h, const double* d, const double* dd) {
  auto* S = static_cast<Sim<Dual>*>(h);
  S->delta.resize(S->ncell);
  for (long c = 0; c < S->ncell; ++c) S->delta[c] = Dual(d ? d[c] : 0.0, dd ? dd[c] : 0.0);
  return 0;
}
int ort_step(void* h, int n) {
  auto* S = static_cast<Sim<Dual>*>(h);
  for (int k = 0; k < n; ++k) S->do_step();
  return 0;
}
int ort_ft(void* h, double* vals, double* tans) {
  auto* S = static_cast<Sim<Dual>*>(h);
  for (size_t k = 0; k < S->ft.size(); ++k) {
    vals[k] = S->ft[k].v;
    tans[k] = S->ft[k].d;
  }
  return (int)S->ft.size();
}
int ort_get_f(void* h, double* vals, double* tans) {
  auto* S = static_cast<Sim<Dual>*>(h);
  S->ensure_state();
  for (size_t k = 0; k < S->f.size(); ++k) {
    vals[k] = S->f[k].v;
    if (tans) tans[k] = S->f[k].d;
  }
  return 0;
}

}  // extern "C"
