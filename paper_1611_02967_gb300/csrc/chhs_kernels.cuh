// chhs_kernels.cuh -- device code of the FAS multigrid solve of one CHHS time
// step (Chen, Feng, Liu, Wang, Wise, arXiv:1611.02967, Section 2, Eqs. 2.4-2.7).
//
// The system solved at every time step, with u = (phi, mu, p) cell-centred:
//   N1(u) = phi - s div_h(M(A_h phi*) grad_h mu) - s div_h(A_h phi* grad_h p) = f_phi
//   N2(u) = mu - chi(phi, phi^m) + (3/4) eps^2 Lap_h phi                    = f_mu
//   N3(u) = -Lap_h p - gamma div_h(A_h phi* grad_h mu)                      = f_p
// On the finest grid f = (phi^m, -phi* - (1/4) eps^2 Lap_h phi^{m-1}, 0); on a
// coarse grid f is the FAS right-hand side R(f - N(u)) + N_c(R u).
//
// Correction form (CORR = true, used by the single-precision inner solves of
// the mixed-precision path): the unknown is a correction e to a base state
// with phi-part phi_b, and chi(phi, phi^m) becomes
//   chi(phi_b + e, phi^m) - chi(phi_b, phi^m)
//     = e (3 phi_b^2 + 2 phi_b phi^m + (phi^m)^2 + (3 phi_b + phi^m) e + e^2) / 4,
// so that N(base + e) - N(base) is evaluated without cancellation; every other
// term of N is linear and keeps its form.
//
// Grid functions are stored x fastest, interior cells only.  The homogeneous
// Neumann ghosts of Appendix A (ghost = mirror of its neighbour) make every
// boundary-face difference vanish, so boundary faces carry no flux and the
// stencil loops below simply skip them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace chhs_dev {

constexpr int kBlock = 256;        // block size of the plain per-cell kernels
constexpr int kSmoothBlock = 128;  // block size of the smoother (more, smaller blocks per SM)
constexpr int kTailThreads = 512;  // one block runs the coarse tail of a V-cycle
constexpr int kTailMaxLevels = 12;

template <typename T>
struct Level {
  T *phi, *mu, *p;     // unknowns (the correction e in correction form)
  T *fphi, *fmu, *fp;  // right-hand sides
  T *phim, *phis;      // phi^m and phi* restricted to this level (fixed in a step)
  T *phib;             // correction form only: phi-part of the base state
  T *phi2, *mu2, *p2;  // 2D single precision only: the tiles' second copy of (phi, mu, p)
  T *fc1, *fc2, *fc3;  // ... and the completed FAS right-hand side (k_tile)
  T *phi0, *mu0, *p0;  // restricted iterate R u kept for the FAS correction
  // Coefficients fixed for a time step (k_coef): a = A_h phi* and M(a) on the
  // +x, +y (+z) face of every cell (zero on boundary faces), their sums over a
  // cell's interior faces, and the smoother's per-cell constants (coef_at).
  T *ax, *ay, *az, *Mx, *My, *Mz;
  T *sM, *sa;
  T *cAe, *cC, *cGn, *cHn, *cQ, *cH;
  int nx, ny, nz;  // nz == 1 in 2D
  int ncell;
  float rnx, rny, rhw;  // 1/nx, 1/ny, 1/ceil(nx/2) in single precision (small_div)
  T ih2, h2;       // 1/h^2 and h^2 on this level
  T sih2;          // s / h^2
  T e34ih2;        // (3/4) eps^2 / h^2
};

template <typename T>
struct Coefs {
  T s;      // time step
  T gamma;  // Darcy coupling, M(x) = 1 + gamma x^2
  T e34;    // (3/4) eps^2
};

// Device-resident bookkeeping of the V-cycle loop of one handle.
struct DevState {
  int vcycles;     // V-cycles of the step in progress
  int vtotal;      // V-cycles summed over the steps of one chhs_step call
  int steps_done;  // steps advanced in that call
  int failed;      // 0, or the chhs_status that stopped the call
  int max_v;
  int go;          // 1 while another V-cycle is due (mirror of the loop condition)
  double tol;
  double tol_max;  // bound of the pointwise guard (infinite when it is off)
  double resid;    // last fine-grid stopping norm
  double rmax;     // last fine-grid pointwise residual max(|r_phi|, |r_mu|, |s r_p|)
  double r0;       // stopping norm at the start of the step
  double pmean;    // mean of p, removed when the step is accepted
  double diag[8];  // reduction results (mass, energies)
  unsigned int ticket;  // blocks of the norm kernel that have finished
  unsigned int pad_;
  // V-cycles between two stopping norms (loop_decision): the iteration about
  // to run does `inner` of them (1 .. max_inner); rho is the measured
  // contraction per V-cycle, rprev the previous norm.
  int inner;
  int go_more[3];  // go and inner >= 2 + q: the batched step's gates of the extra V-cycles
  int max_inner;   // 0 or 1: a norm after every V-cycle
  int checks;      // stopping norms after V-cycles in the current call
  int use_if;      // IF nodes of cond_if in the step graph (0 .. 3)
  double rho;
  double rprev;
  cudaGraphConditionalHandle cond_if[3];  // IF node q: a (2 + q)-th V-cycle in the iteration
};

// Most V-cycles between two stopping norms (DevState::go_more, cond_if hold kMaxInner - 1).
constexpr int kMaxInner = 4;

// chi(a, b) = (a^2 + b^2)(a + b) / 4 (Eq. 2.4) and d chi / d a.
template <typename T>
__device__ __forceinline__ T chi(T a, T b) { return T(0.25) * (a * a + b * b) * (a + b); }
template <typename T>
__device__ __forceinline__ T dchi_da(T a, T b) { return T(0.25) * (T(3) * a * a + T(2) * a * b + b * b); }

// The nonlinear term of N2 at cell c for the unknown value v, and its
// derivative in v (plain form, or correction form around phi_b).
template <typename T, bool CORR>
__device__ __forceinline__ T chi_term(const Level<T>& L, int c, T v, T pm) {
  if (CORR) {
    T b = L.phib[c];
    return T(0.25) * v * (T(3) * b * b + T(2) * b * pm + pm * pm + (T(3) * b + pm) * v + v * v);
  }
  return chi(v, pm);
}
template <typename T, bool CORR>
__device__ __forceinline__ T dchi_term(const Level<T>& L, int c, T v, T pm) {
  return CORR ? dchi_da(L.phib[c] + v, pm) : dchi_da(v, pm);
}

// Approximate reciprocal of x >= 1 (the PTX rcp.approx instruction).  It
// scales the smoother's local Newton update only: an inexact local Jacobian
// changes how fast the sweep contracts, never its fixed point (zero residual).
__device__ __forceinline__ double rcp_approx(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// n (exactly) and 1/n (to single precision) for the interior-face count n in
// 1..6.  A chain of selections between constants was measured to cost ~430
// cycles per use (an indexed constant-table load); these are a few integer
// or single-precision instructions.  The double n is assembled from its bits
// (exponent floor(log2 n), mantissa n shifted into place), so no FP64-pipe
// conversion is spent on it.  1/n only scales smoother updates and stored
// Jacobian constants (never a term of a residual), so single precision
// suffices (the hardware reciprocal approximation in single-precision code).
template <typename T>
__device__ __forceinline__ T count_value(int n);
template <>
__device__ __forceinline__ float count_value<float>(int n) { return (float)n; }
template <>
__device__ __forceinline__ double count_value<double>(int n) {
  const int e = 31 - __clz(n);
  const unsigned hi = ((unsigned)(1023 + e) << 20) | (((unsigned)n << (20 - e)) & 0xFFFFFu);
  return __hiloint2double((int)hi, 0);
}
template <typename T>
__device__ __forceinline__ T inv_count(int n) { return T(__frcp_rn((float)n)); }
template <>
__device__ __forceinline__ float inv_count<float>(int n) { return rcp_approx((float)n); }

// Programmatic dependent launch: the kernels of a step are launched so that
// each may be scheduled while its predecessor drains (its blocks trigger the
// launch implicitly when they exit), and each first waits until the
// predecessor grid has completed and its writes are visible.  No block
// triggers early, so a successor's blocks are never placed on the SMs before
// its predecessor has finished issuing work (an early trigger unbalanced the
// large grids).
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void cell_ijk(int c, int nx, int ny, int& i, int& j, int& k) {
  i = c % nx;
  int r = c / nx;
  j = r % ny;
  k = r / ny;
}

// t / d for 0 <= t < 2^21 and d >= 1, given rd = 1/d rounded to single
// precision: (t + 1/2) / d lies at least 1/(2d) from an integer, and the
// product (t + 1/2) * rd errs by less than 2^-22 (t + 1/2) / d, which is
// smaller for t < 2^21, so truncation gives the exact quotient.  Two
// single-precision operations instead of an integer division.
__device__ __forceinline__ int small_div(int t, float rd) { return __float2int_rz((float(t) + 0.5f) * rd); }

// cell_ijk for levels of fewer than 2^21 cells (the tail's levels).
template <typename T>
__device__ __forceinline__ void cell_ijk_small(int c, const Level<T>& L, int& i, int& j, int& k) {
  const int r = small_div(c, L.rnx);
  i = c - r * L.nx;
  k = small_div(r, L.rny);
  j = r - k * L.ny;
}

// Neighbour sums of one cell over its interior faces f (neighbour e):
//   Mp = sum (M_f mu_e + a_f p_e), amu = sum a_f mu_e,
//   phi = sum phi_e, p = sum p_e, m = n_c.
// With sM = sum M_f and sa = sum a_f (k_coef), the face sums of N become
//   sum M_f (mu_e - mu_c) + a_f (p_e - p_c) = Mp - sM mu_c - sa p_c, ...
// The plain sums start from -0 (x + -0 = x exactly), so the compiler drops
// the first addition.
// Double to single precision with integer instructions, truncating toward
// zero: a conversion instruction costs as much as an FP64 FMA on this GPU
// (measured), these are a handful of integer operations.  For the values it
// sees (residuals and phi, far inside the single-precision range) the result
// is x with its mantissa cut to 24 bits (relative error below 2^-23);
// magnitudes under the smallest normal single give 0 and ones beyond its
// range give infinity.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned bits = e <= 0 ? sign : e >= 255 ? (sign | 0x7F800000u) : (sign | ((unsigned)e << 23) | mant);
  return __uint_as_float(bits);
}

// Single to double precision with integer instructions, exactly (the
// inverse direction of f64_to_f32_rz): exponent rebiased, mantissa moved
// into place.  Zeros and subnormal singles give a signed zero, infinities
// and NaNs stay infinities and NaNs.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned mant = b & 0x7FFFFFu;
  const unsigned hi = e == 0u ? sign
                      : e == 255u ? (sign | 0x7FF00000u | (mant >> 3) | (mant ? 0x80000u : 0u))
                                  : (sign | ((e + 896u) << 20) | (mant >> 3));
  const unsigned lo = (e == 0u || e == 255u) ? 0u : (mant << 29);
  return __hiloint2double((int)hi, (int)lo);
}

template <typename T>
struct Nb {
  T Mp, amu, phi, p;
  int m;
};

template <typename T, int DIM>
__device__ __forceinline__ void nb_sums(const Level<T>& L, const T* phi, const T* mu, const T* p, int c,
                                        int i, int j, int k, Nb<T>& S) {
  S.Mp = S.amu = S.phi = S.p = T(-0.0);
  S.m = 0;
  // Branch-free: a missing face reads cell c itself (a valid index) and
  // contributes a = M = 0 and -0 to the plain sums, so all loads of a cell
  // issue together.  The face coefficient of face f between c and e is held
  // by the lower of the two cells (fe).
  auto face = [&](bool in, int e, int fe, const T* af, const T* Mf) {
    const int es = in ? e : c, fs = in ? fe : c;
    const T mue = mu[es], pe = p[es], phie = phi[es], a0 = af[fs], M0 = Mf[fs];
    const T a = in ? a0 : T(0), M = in ? M0 : T(0);
    S.Mp += M * mue;
    S.Mp += a * pe;
    S.amu += a * mue;
    S.phi += in ? phie : T(-0.0);
    S.p += in ? pe : T(-0.0);
    S.m += in ? 1 : 0;
  };
  const int sy = L.nx, sz = L.nx * L.ny;
  face(i > 0, c - 1, c - 1, L.ax, L.Mx);
  face(i + 1 < L.nx, c + 1, c, L.ax, L.Mx);
  face(j > 0, c - sy, c - sy, L.ay, L.My);
  face(j + 1 < L.ny, c + sy, c, L.ay, L.My);
  if (DIM == 3) {
    face(k > 0, c - sz, c - sz, L.az, L.Mz);
    face(k + 1 < L.nz, c + sz, c, L.az, L.Mz);
  }
}

// The cubic of the plain form's N2 in the cell's own phi = v:
//   P(v) = chi(v, pm) - pm^3/4 + (3/4) eps^2 n_c v / h^2
//        = ((v/4 + pm/4) v + Q) v,   Q = pm^2/4 + (3/4) eps^2 n_c / h^2 (coef_at),
// and B = P'(v) = (3v/4 + pm/2) v + Q.  The plain form carries N2 + pm^3/4
// and f_mu + pm^3/4 (k_setup_coef) instead of N2 and f_mu: the residual
// f_mu - N2, the FAS coarse right-hand sides R r + N_c(R u) and the
// corrections they drive are the same, and each evaluation saves the
// constant term.
template <typename T>
__device__ __forceinline__ T cubic_P(T v, T hp, T Q) { return ((T(0.25) * v + hp) * v + Q) * v; }

// N(u) at cell c for the fields (phi, mu, p) given explicitly (plain form:
// N2 shifted by pm^3/4, see cubic_P).
template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void eval_N(const Level<T>& L, const Coefs<T>& K, const T* phi, const T* mu,
                                       const T* p, int c, int i, int j, int k, T& n1, T& n2, T& n3) {
  Nb<T> S;
  nb_sums<T, DIM>(L, phi, mu, p, c, i, j, k, S);
  T phic = phi[c], muc = mu[c], pc = p[c];
  T sM = L.sM[c], sa = L.sa[c], mm = count_value<T>(S.m);
  n1 = phic - L.sih2 * ((S.Mp - sM * muc) - sa * pc);
  if (CORR)
    n2 = muc - chi_term<T, CORR>(L, c, phic, L.phim[c]) + L.e34ih2 * (S.phi - mm * phic);
  else
    n2 = (muc + L.e34ih2 * S.phi) - cubic_P(phic, L.cH[c], L.cQ[c]);
  n3 = -L.ih2 * ((S.p - mm * pc) + K.gamma * (S.amu - sa * muc));
}

// Coefficients of a time step at cell c of one level, from phi*: the face
// values a_f = (phi*_c + phi*_e)/2 and M_f = 1 + gamma a_f^2 on the
// +x/+y/+z faces, sM = sum M_f and sa = sum a_f over the interior faces, and
// the smoother's constants (cell_update)
//   Ae = (s/h^2)(sM - gamma sa^2 / n_c),  C = s sa / h^2,  G/Dn = gamma sa / n_c,
//   1/Dn = h^2 / n_c,  Q = pm^2/4 + (3/4) eps^2 n_c / h^2,  and pm/4.
// ps(e) returns phi* at cell e; pmc is phi^m at c.
template <typename T, int DIM, class PS>
__device__ __forceinline__ void coef_at(const Level<T>& L, const Coefs<T>& K, int c, int i, int j, int k,
                                        PS ps, T pmc) {
  const T pc = ps(c);
  T sumM = 0, suma = 0;
  int m = 0;
  auto face = [&](int e, T* a_out, T* M_out) {
    T a = T(0.5) * (pc + ps(e));
    T M = T(1) + K.gamma * a * a;
    sumM += M;
    suma += a;
    m += 1;
    if (a_out) {
      a_out[c] = a;
      M_out[c] = M;
    }
  };
  const int sy = L.nx, sz = L.nx * L.ny;
  if (i > 0) face(c - 1, nullptr, nullptr);
  if (i + 1 < L.nx) face(c + 1, L.ax, L.Mx);
  else L.ax[c] = L.Mx[c] = T(0);
  if (j > 0) face(c - sy, nullptr, nullptr);
  if (j + 1 < L.ny) face(c + sy, L.ay, L.My);
  else L.ay[c] = L.My[c] = T(0);
  if (DIM == 3) {
    if (k > 0) face(c - sz, nullptr, nullptr);
    if (k + 1 < L.nz) face(c + sz, L.az, L.Mz);
    else L.az[c] = L.Mz[c] = T(0);
  }
  T im = inv_count<T>(m);
  L.sM[c] = sumM;
  L.sa[c] = suma;
  L.cAe[c] = L.sih2 * (sumM - K.gamma * suma * suma * im);
  L.cC[c] = L.sih2 * suma;
  L.cGn[c] = K.gamma * suma * im;
  L.cHn[c] = L.h2 * im;
  L.cQ[c] = T(0.25) * pmc * pmc + L.e34ih2 * count_value<T>(m);
  L.cH[c] = T(0.25) * pmc;
}

// phi^m and phi* of the 2^d-cell block whose corner is (i, j, k), restricted
// (mean of the children) into the next coarser level; pm(e), ps(e) give the
// fine values.
template <typename T, typename U, int DIM, class PM, class PS>
__device__ __forceinline__ void restrict_coef_at(const Level<U>& F, const Level<T>& C, int i, int j, int k,
                                                 PM pm, PS ps) {
  T a = 0, b = 0;
  const int kz = DIM == 3 ? 2 : 1;
  for (int dk = 0; dk < kz; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int e = (i + di) + F.nx * ((j + dj) + F.ny * (k + dk));
        a += pm(e);
        b += ps(e);
      }
  const T w = DIM == 3 ? T(0.125) : T(0.25);
  int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
  C.phim[q] = w * a;
  C.phis[q] = w * b;
}

// A level's coefficients, and the restriction of phi^m and phi* to the next
// level (has_next), in one pass.
template <typename T, int DIM>
__device__ __forceinline__ void coef_restrict_body(int bx, Level<T> L, Coefs<T> K, Level<T> Cn, int has_next) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= L.ncell) return;
  int i, j, k;
  cell_ijk(c, L.nx, L.ny, i, j, k);
  auto ps = [&](int e) { return L.phis[e]; };
  auto pm = [&](int e) { return L.phim[e]; };
  coef_at<T, DIM>(L, K, c, i, j, k, ps, pm(c));
  if (has_next && !(i & 1) && !(j & 1) && (DIM == 2 || !(k & 1))) restrict_coef_at<T, T, DIM>(L, Cn, i, j, k, pm, ps);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_coef_restrict(Level<T> L, Coefs<T> K, Level<T> Cn, int has_next) {
  pdl_enter();
  coef_restrict_body<T, DIM>(blockIdx.x, L, K, Cn, has_next);
}

// ---------------------------------------------------------------- smoother
//
// One colour pass of red-black nonlinear Gauss-Seidel.  Cells of one colour
// only couple to cells of the other, so every cell of the colour is updated
// at once.  The update is one Newton step on the cell's own (phi, mu, p) with
// its neighbours frozen; eliminating the cell's own pressure equation leaves
// a 2x2 Newton system in (phi, mu):
//   A  = s sum M_f / h^2,  C = s sum a_f / h^2,  G = gamma sum a_f / h^2,
//   Dn = n_c / h^2,        B = chi_a(phi, phi^m) + (3/4) eps^2 n_c / h^2,
//   Ae = A - C G / Dn = (s/h^2)(sum M_f - gamma (sum a_f)^2 / n_c) >= s n_c / h^2,
//   dphi = (R1 - Ae R2 - C (R3/Dn)) / (1 + Ae B),  dmu = R2 + B dphi,
//   dp = R3/Dn - (G/Dn) dmu,
// with R = f - N(u) at the cell.  R3 is formed as the residual itself and
// then scaled by 1/Dn = h^2/n_c (a stored constant that may be inexact: it
// only scales the update, while an inexact factor applied before the
// subtraction of n_c p_c would move the smoother's fixed point).
// The constants Ae, C, G/Dn, 1/Dn and Q (B = P'(phi), cubic_P) come from
// coef_at; chi_a in the correction form is taken at phi_b + e.
//
// In the plain double-precision form the residuals R and the update of the
// state are double precision, while the 2x2 solve that turns R into the
// step (B, 1/(1 + Ae B) and the products with the constants) runs in single
// precision (newton_step_f32): it only scales the step, so the sweep's fixed
// point -- zero residual -- is the double-precision one, and the step it
// takes differs from the exact Newton step by ~1e-7 of its length.  On
// GB300 this removes a quarter of the cell's FP64-pipe instructions.
struct StepF32 {
  float dphi, dmu, dp;
};

// The 2x2 Newton solve in single precision from the double-precision
// residuals R1, R2, R3 (R3 not yet scaled by 1/Dn) and B's terms t, t2 at
// the cell's phi (cell_update); the Jacobian constants are cut to single
// precision with integer instructions.
__device__ __forceinline__ StepF32 newton_step_f32(double R1, double R2, double R3, double phic, double t,
                                                   double t2, double Ae, double cC, double cGn, double cHn) {
  const float v = f64_to_f32_rz(phic), tf = f64_to_f32_rz(t), t2f = f64_to_f32_rz(t2);
  const float B = (0.25f * v + tf) * v + t2f;
  const float ae = f64_to_f32_rz(Ae);
  const float r2 = f64_to_f32_rz(R2);
  const float r3n = f64_to_f32_rz(cHn) * f64_to_f32_rz(R3);
  StepF32 d;
  d.dphi = ((f64_to_f32_rz(R1) - ae * r2) - f64_to_f32_rz(cC) * r3n) * rcp_approx(1.f + ae * B);
  d.dmu = r2 + B * d.dphi;
  d.dp = r3n - f64_to_f32_rz(cGn) * d.dmu;
  return d;
}

template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void cell_update(const Level<T>& L, const Coefs<T>& K, int c, int i, int j,
                                            int k, T f1, T f2, T f3) {
  Nb<T> S;
  nb_sums<T, DIM>(L, L.phi, L.mu, L.p, c, i, j, k, S);
  T phic = L.phi[c], muc = L.mu[c], pc = L.p[c];
  T sM = L.sM[c], sa = L.sa[c], Q = L.cQ[c];
  T hp = L.cH[c];
  T R1 = (f1 - phic) + L.sih2 * ((S.Mp - sM * muc) - sa * pc);
  T R2, B, t = T(0), t2 = T(0);
  if (CORR) {
    R2 = f2 - muc + chi_term<T, CORR>(L, c, phic, L.phim[c]) - L.e34ih2 * (S.phi - count_value<T>(S.m) * phic);
    const T w = L.phib[c] + phic;
    B = (T(0.75) * w + (hp + hp)) * w + Q;
  } else {
    // cubic_P(v) = t2 v with t = v/4 + pm/4, t2 = t v + Q; P'(v) = (t + v/4) v + t2
    t = T(0.25) * phic + hp;
    t2 = t * phic + Q;
    R2 = ((f2 - muc) - L.e34ih2 * S.phi) + t2 * phic;
    B = (T(0.25) * phic + t) * phic + t2;
  }
  const T R3 = f3 + L.ih2 * ((S.p - count_value<T>(S.m) * pc) + K.gamma * (S.amu - sa * muc));
  if constexpr (sizeof(T) == 8 && !CORR) {
    const StepF32 d = newton_step_f32(R1, R2, R3, phic, t, t2, L.cAe[c], L.cC[c], L.cGn[c], L.cHn[c]);
    L.phi[c] = phic + f32_to_f64_exact(d.dphi);
    L.mu[c] = muc + f32_to_f64_exact(d.dmu);
    L.p[c] = pc + f32_to_f64_exact(d.dp);
  } else {
    T R3n = L.cHn[c] * R3;
    T Ae = L.cAe[c];
    T dphi = ((R1 - Ae * R2) - L.cC[c] * R3n) * rcp_approx(T(1) + Ae * B);
    T dmu = R2 + B * dphi;
    T dp = R3n - L.cGn[c] * dmu;
    L.phi[c] = phic + dphi;
    L.mu[c] = muc + dmu;
    L.p[c] = pc + dp;
  }
}

// The right-hand side at cell c for a smoothing pass.  With rhs set (the
// first pre-smoothing sweep on a coarse level) it first completes the FAS
// right-hand side f_c = R r + N_c(R u) from the saved R u (phi0, mu0, p0).
template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void cell_rhs(const Level<T>& L, const Coefs<T>& K, int c, int i, int j, int k,
                                         bool rhs, T& f1, T& f2, T& f3) {
  f1 = L.fphi[c];
  f2 = L.fmu[c];
  f3 = L.fp[c];
  if (rhs) {
    T n1, n2, n3;
    eval_N<T, DIM, CORR>(L, K, L.phi0, L.mu0, L.p0, c, i, j, k, n1, n2, n3);
    f1 += n1;
    f2 += n2;
    f3 += n3;
    L.fphi[c] = f1;
    L.fmu[c] = f2;
    L.fp[c] = f3;
  }
}

// Threads cover only the cells of the colour: ceil(nx/2) per grid row, the
// row's first cell of the colour at i = (j + k + colour) & 1.
template <typename T, int DIM, bool CORR>
__global__ void __launch_bounds__(kSmoothBlock) k_smooth(Level<T> L, Coefs<T> K, int colour, int rhs) {
  pdl_enter();
  const int hw = (L.nx + 1) >> 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int row, k;
  if (t < (1 << 21)) {
    row = small_div(t, L.rhw);
    k = small_div(row, L.rny);
  } else {
    row = t / hw;
    k = row / L.ny;
  }
  const int ti = t - row * hw, j = row - k * L.ny;
  if (k >= L.nz) return;
  int i = 2 * ti + ((j + k + colour) & 1);
  if (i >= L.nx) return;
  int c = i + L.nx * (j + L.ny * k);
  T f1, f2, f3;
  cell_rhs<T, DIM, CORR>(L, K, c, i, j, k, rhs != 0, f1, f2, f3);
  cell_update<T, DIM, CORR>(L, K, c, i, j, k, f1, f2, f3);
}

// ---------------------------------------------------------------- split update
//
// On small double-precision levels a colour pass is one warp's chain of FP64
// instructions, and each FP64 warp instruction holds its sub-partition's
// FP64 pipe for ~64 cycles however few lanes are live.  So the update of a
// cell is split over the three warps of a group (three sub-partitions, three
// FP64 pipes): warp 0 forms R1 (and the phi row of the FAS right-hand side),
// warp 1 R3/Dn (pressure row), warp 2 R2, B and 1/(1 + Ae B) (mu row); warps
// 1 and 2 hand their values over through shared memory and warp 0 finishes
// the update.  Same formulas as cell_update, plain form only.
//
// The face loop of the split update: for every face of cell c, in the order
// of nb_sums, fn(in, es, fs) with the neighbour es and face-coefficient
// index fs (both c itself for a missing face).
template <int DIM, class FN>
__device__ __forceinline__ void for_faces(const Level<double>& L, int c, int i, int j, int k, FN fn) {
  const int sy = L.nx, sz = L.nx * L.ny;
  auto f = [&](bool in, int e, int fe, int dir) { fn(in, in ? e : c, in ? fe : c, dir); };
  f(i > 0, c - 1, c - 1, 0);
  f(i + 1 < L.nx, c + 1, c, 0);
  f(j > 0, c - sy, c - sy, 1);
  f(j + 1 < L.ny, c + sy, c, 1);
  if (DIM == 3) {
    f(k > 0, c - sz, c - sz, 2);
    f(k + 1 < L.nz, c + sz, c, 2);
  }
}

// x: this lane's four exchange slots, stride 32.  bar() synchronises the
// three warps of the group; every warp of the group calls this the same
// number of times (act may be false).  As in cell_update, the residual rows
// are double precision and the 2x2 solve is single precision: warp 1 hands
// over R3/Dn, warp 2 R2, B and 1/(1 + Ae B), all in single precision.
template <int DIM, class BAR>
__device__ __forceinline__ void cell_update_split(const Level<double>& L, const Coefs<double>& K, int role,
                                                  bool act, int c, int i, int j, int k, bool rhs, float* x,
                                                  BAR bar) {
  const double* af[3] = {L.ax, L.ay, L.az};
  const double* Mf[3] = {L.Mx, L.My, L.Mz};
  double R1 = 0.0, phic = 0.0, muc = 0.0, pc = 0.0, Ae = 0.0, cC = 0.0, cGn = 0.0;
  if (act) {
    const double sa = L.sa[c];
    if (role == 0) {
      double Mp = -0.0;
      for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
        const double a0 = af[d][fs], M0 = Mf[d][fs], mue = L.mu[es], pe = L.p[es];
        const double a = in ? a0 : 0.0, M = in ? M0 : 0.0;
        Mp += M * mue;
        Mp += a * pe;
      });
      phic = L.phi[c];
      muc = L.mu[c];
      pc = L.p[c];
      Ae = L.cAe[c];
      cC = L.cC[c];
      cGn = L.cGn[c];
      const double sM = L.sM[c];
      double f1 = L.fphi[c];
      if (rhs) {
        double Mp0 = -0.0;
        for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
          const double a0 = af[d][fs], M0 = Mf[d][fs], mue = L.mu0[es], pe = L.p0[es];
          const double a = in ? a0 : 0.0, M = in ? M0 : 0.0;
          Mp0 += M * mue;
          Mp0 += a * pe;
        });
        f1 += L.phi0[c] - L.sih2 * ((Mp0 - sM * L.mu0[c]) - sa * L.p0[c]);
        L.fphi[c] = f1;
      }
      R1 = (f1 - phic) + L.sih2 * ((Mp - sM * muc) - sa * pc);
    } else if (role == 1) {
      double amu = -0.0, sp = -0.0;
      int m = 0;
      for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
        const double a0 = af[d][fs], mue = L.mu[es], pe = L.p[es];
        const double a = in ? a0 : 0.0;
        amu += a * mue;
        sp += in ? pe : -0.0;
        m += in ? 1 : 0;
      });
      const double mm = count_value<double>(m);
      double f3 = L.fp[c];
      if (rhs) {
        double amu0 = -0.0, sp0 = -0.0;
        for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
          const double a0 = af[d][fs], mue = L.mu0[es], pe = L.p0[es];
          const double a = in ? a0 : 0.0;
          amu0 += a * mue;
          sp0 += in ? pe : -0.0;
        });
        f3 += -L.ih2 * ((sp0 - mm * L.p0[c]) + K.gamma * (amu0 - sa * L.mu0[c]));
        L.fp[c] = f3;
      }
      const double R3 = f3 + L.ih2 * ((sp - mm * L.p[c]) + K.gamma * (amu - sa * L.mu[c]));
      x[0] = f64_to_f32_rz(L.cHn[c]) * f64_to_f32_rz(R3);
    } else {
      double sphi = -0.0;
      for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
        const double ph = L.phi[es];
        sphi += in ? ph : -0.0;
      });
      const double v = L.phi[c], Q = L.cQ[c], hp = L.cH[c];
      double f2 = L.fmu[c];
      if (rhs) {
        double sphi0 = -0.0;
        for_faces<DIM>(L, c, i, j, k, [&](bool in, int es, int fs, int d) {
          const double ph = L.phi0[es];
          sphi0 += in ? ph : -0.0;
        });
        f2 += (L.mu0[c] + L.e34ih2 * sphi0) - cubic_P(L.phi0[c], hp, Q);
        L.fmu[c] = f2;
      }
      const double t = 0.25 * v + hp;
      const double t2 = t * v + Q;
      const double R2 = ((f2 - L.mu[c]) - L.e34ih2 * sphi) + t2 * v;
      const float vf = f64_to_f32_rz(v);
      const float B = (0.25f * vf + f64_to_f32_rz(t)) * vf + f64_to_f32_rz(t2);
      x[32] = f64_to_f32_rz(R2);
      x[64] = B;
      x[96] = rcp_approx(1.f + f64_to_f32_rz(L.cAe[c]) * B);
    }
  }
  bar();
  if (act && role == 0) {
    const float R3n = x[0], R2 = x[32], B = x[64], rd = x[96];
    const float ae = f64_to_f32_rz(Ae);
    const float dphi = ((f64_to_f32_rz(R1) - ae * R2) - f64_to_f32_rz(cC) * R3n) * rd;
    const float dmu = R2 + B * dphi;
    const float dp = R3n - f64_to_f32_rz(cGn) * dmu;
    L.phi[c] = phic + f32_to_f64_exact(dphi);
    L.mu[c] = muc + f32_to_f64_exact(dmu);
    L.p[c] = pc + f32_to_f64_exact(dp);
  }
}

// Colour pass of a small double-precision level with the split update: one
// group of three warps (96 threads) per 32 cells of the colour.
template <int DIM>
__global__ void __launch_bounds__(96) k_smooth_split(Level<double> L, Coefs<double> K, int colour, int rhs) {
  pdl_enter();
  __shared__ float xch[4 * 32];
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int hw = (L.nx + 1) >> 1;
  const int t = blockIdx.x * 32 + lane;
  int row, k;
  if (t < (1 << 21)) {
    row = small_div(t, L.rhw);
    k = small_div(row, L.rny);
  } else {
    row = t / hw;
    k = row / L.ny;
  }
  const int ti = t - row * hw, j = row - k * L.ny;
  const int i = 2 * ti + ((j + k + colour) & 1);
  const bool act = k < L.nz && i < L.nx;
  const int c = act ? i + L.nx * (j + L.ny * k) : 0;
  cell_update_split<DIM>(L, K, role, act, c, i, j, k, rhs != 0, xch + lane, [] { __syncthreads(); });
}

// f_c += N_c(R u) on every cell (used when there is no pre-smoothing sweep to
// carry it).
template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void coarse_rhs_body(int bx, Level<T> C, Coefs<T> K) {
  int q = bx * blockDim.x + threadIdx.x;
  if (q >= C.ncell) return;
  int i, j, k;
  cell_ijk(q, C.nx, C.ny, i, j, k);
  T f1, f2, f3;
  cell_rhs<T, DIM, CORR>(C, K, q, i, j, k, true, f1, f2, f3);
}

template <typename T, int DIM, bool CORR>
__global__ void __launch_bounds__(kBlock) k_coarse_rhs(Level<T> C, Coefs<T> K) {
  pdl_enter();
  coarse_rhs_body<T, DIM, CORR>(blockIdx.x, C, K);
}

// ---------------------------------------------------------------- transfers

// Residual and restriction, one thread per fine cell.  A warp covers a tile
// of 16 x 2 (2D) or 8 x 2 x 2 (3D) fine cells, so the 2^d children of a
// coarse cell sit in lanes l, l^1, l^16 (2D) or l, l^1, l^8, l^16 (3D) and are
// summed by shuffles.  Writes u_c = R u (twice: the coarse iterate and u_c^0),
// R phi_b in correction form, and f_c = R r (completed later by N_c(R u)).
template <typename T, int DIM, bool CORR>
__global__ void __launch_bounds__(kBlock) k_residual_restrict(Level<T> F, Level<T> C, Coefs<T> K) {
  pdl_enter();
  constexpr int TX = DIM == 3 ? 8 : 16;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tiles_x = (F.nx + TX - 1) / TX;
  const int tiles_y = F.ny >> 1;
  const int tiles_z = DIM == 3 ? (F.nz >> 1) : 1;
  if (warp >= tiles_x * tiles_y * tiles_z) return;  // whole warp
  const int tx = warp % tiles_x;
  const int rest = warp / tiles_x;
  const int ty = rest % tiles_y, tz = rest / tiles_y;
  const int i = tx * TX + (lane % TX);
  const int j = 2 * ty + ((lane / TX) & 1);
  const int k = DIM == 3 ? 2 * tz + (lane >> 4) : 0;
  const bool valid = i < F.nx;
  constexpr int NV = CORR ? 7 : 6;
  T v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = T(0);
  if (valid) {
    int c = i + F.nx * (j + F.ny * k);
    T n1, n2, n3;
    eval_N<T, DIM, CORR>(F, K, F.phi, F.mu, F.p, c, i, j, k, n1, n2, n3);
    v[0] = F.fphi[c] - n1;
    v[1] = F.fmu[c] - n2;
    v[2] = F.fp[c] - n3;
    v[3] = F.phi[c];
    v[4] = F.mu[c];
    v[5] = F.p[c];
    if (CORR) v[NV - 1] = F.phib[c];
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1);
    v[q] += __shfl_xor_sync(0xffffffffu, v[q], TX);
    if (DIM == 3) v[q] += __shfl_xor_sync(0xffffffffu, v[q], 16);
  }
  const bool leader = valid && (lane & 1) == 0 && ((lane / TX) & 1) == 0 && (DIM == 2 || lane < 16);
  if (!leader) return;
  const T w = DIM == 3 ? T(0.125) : T(0.25);
  int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
  C.fphi[q] = w * v[0];
  C.fmu[q] = w * v[1];
  C.fp[q] = w * v[2];
  C.phi[q] = C.phi0[q] = w * v[3];
  C.mu[q] = C.mu0[q] = w * v[4];
  C.p[q] = C.p0[q] = w * v[5];
  if (CORR) C.phib[q] = w * v[NV - 1];
}

// One row of the plain form's N at cell c, on the fields (phi, mu, p):
// role 0 gives N1, role 1 N3, role 2 N2 (eval_N's formulas, one row each, so
// three warps can share a cell's work).  u returns the row's own unknown at c
// (phi, p or mu).  f_row gives the matching right-hand side.
template <int DIM>
__device__ __forceinline__ double n_row(const Level<double>& F, const Coefs<double>& K, int role,
                                        const double* phi, const double* mu, const double* p, int c, int i,
                                        int j, int k, double& u) {
  const double* af[3] = {F.ax, F.ay, F.az};
  const double* Mf[3] = {F.Mx, F.My, F.Mz};
  const double sa = F.sa[c];
  if (role == 0) {
    double Mp = -0.0;
    for_faces<DIM>(F, c, i, j, k, [&](bool in, int es, int fs, int d) {
      const double a0 = af[d][fs], M0 = Mf[d][fs], mue = mu[es], pe = p[es];
      const double a = in ? a0 : 0.0, M = in ? M0 : 0.0;
      Mp += M * mue;
      Mp += a * pe;
    });
    u = phi[c];
    return u - F.sih2 * ((Mp - F.sM[c] * mu[c]) - sa * p[c]);
  }
  if (role == 1) {
    double amu = -0.0, sp = -0.0;
    int m = 0;
    for_faces<DIM>(F, c, i, j, k, [&](bool in, int es, int fs, int d) {
      const double a0 = af[d][fs], mue = mu[es], pe = p[es];
      const double a = in ? a0 : 0.0;
      amu += a * mue;
      sp += in ? pe : -0.0;
      m += in ? 1 : 0;
    });
    u = p[c];
    return -F.ih2 * ((sp - count_value<double>(m) * u) + K.gamma * (amu - sa * mu[c]));
  }
  double sphi = -0.0;
  for_faces<DIM>(F, c, i, j, k, [&](bool in, int es, int fs, int d) {
    const double ph = phi[es];
    sphi += in ? ph : -0.0;
  });
  u = mu[c];
  return (u + F.e34ih2 * sphi) - cubic_P(phi[c], F.cH[c], F.cQ[c]);
}
__device__ __forceinline__ double* f_row(const Level<double>& F, int role) {
  return role == 0 ? F.fphi : role == 1 ? F.fp : F.fmu;
}

// k_residual_restrict for small double-precision levels (plain form): the
// three warps of a block take the phi, pressure and mu rows of the same
// 16 x 2 (8 x 2 x 2) tile, so each warp's FP64 chain is a third as long.
// Each row's coarse values depend on that row only, so the warps need no
// exchange: warp 0 writes f_phi and phi (phi^0), warp 1 f_p and p (p^0),
// warp 2 f_mu and mu (mu^0).  Same formulas as eval_N.
template <int DIM>
__global__ void __launch_bounds__(96) k_residual_restrict_split(Level<double> F, Level<double> C,
                                                                Coefs<double> K) {
  pdl_enter();
  constexpr int TX = DIM == 3 ? 8 : 16;
  const int lane = threadIdx.x & 31, role = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int tiles_x = (F.nx + TX - 1) / TX;
  const int tiles_y = F.ny >> 1;
  const int tx = tile % tiles_x;
  const int rest = tile / tiles_x;
  const int ty = rest % tiles_y, tz = rest / tiles_y;
  const int i = tx * TX + (lane % TX);
  const int j = 2 * ty + ((lane / TX) & 1);
  const int k = DIM == 3 ? 2 * tz + (lane >> 4) : 0;
  const bool valid = i < F.nx;
  double r = 0.0, u = 0.0;
  if (valid) {
    const int c = i + F.nx * (j + F.ny * k);
    const double n = n_row<DIM>(F, K, role, F.phi, F.mu, F.p, c, i, j, k, u);
    r = f_row(F, role)[c] - n;
  }
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  u += __shfl_xor_sync(0xffffffffu, u, 1);
  r += __shfl_xor_sync(0xffffffffu, r, TX);
  u += __shfl_xor_sync(0xffffffffu, u, TX);
  if (DIM == 3) {
    r += __shfl_xor_sync(0xffffffffu, r, 16);
    u += __shfl_xor_sync(0xffffffffu, u, 16);
  }
  const bool leader = valid && (lane & 1) == 0 && ((lane / TX) & 1) == 0 && (DIM == 2 || lane < 16);
  if (!leader) return;
  const double w = DIM == 3 ? 0.125 : 0.25;
  const int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
  if (role == 0) {
    C.fphi[q] = w * r;
    C.phi[q] = C.phi0[q] = w * u;
  } else if (role == 1) {
    C.fp[q] = w * r;
    C.p[q] = C.p0[q] = w * u;
  } else {
    C.fmu[q] = w * r;
    C.mu[q] = C.mu0[q] = w * u;
  }
}

// u += P(u_c - u_c^0), P piecewise constant.
template <typename T, int DIM>
__device__ __forceinline__ void prolong_body(int bx, Level<T> F, Level<T> C) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= F.ncell) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (DIM == 3 ? (k >> 1) : 0));
  F.phi[c] += C.phi[q] - C.phi0[q];
  F.mu[c] += C.mu[q] - C.mu0[q];
  F.p[c] += C.p[q] - C.p0[q];
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong(Level<T> F, Level<T> C) {
  pdl_enter();
  prolong_body<T, DIM>(blockIdx.x, F, C);
}

// ---------------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV values per thread; thread 0 returns the totals.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = lane < nw ? sh[q][lane] : 0.0;
      v[q] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Sum the partials in a fixed order (deterministic), one block.  Loads go
// through L2 (other blocks of this kernel may have just written them).
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int nparts, double (&tot)[NV]) {
  for (int q = 0; q < NV; ++q) tot[q] = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int q = 0; q < NV; ++q) tot[q] += __ldcg(partials + b * NV + q);
  block_sum<NV>(tot);
}

// The loop decision after a norm r and a pointwise residual rmax.  mode 0:
// start of a step (records r0); mode 1: after a V-cycle (counts it).  The
// step is converged when r <= tol and rmax <= tol_max.  Returns 1 while
// another cycle is due.
// V-cycles for the next iteration of the step's loop: the number the
// measured contraction rho predicts the norms (r against tol, the pointwise
// rmax against tol_max) still need, rounded to the nearest (a V-cycle past
// the stopping point needs a contraction twice as strong, in log terms, as
// the one measured over the iteration before; rounding down instead cost
// ~0.8 more norms per step and no fewer V-cycles on the benchmark
// workloads); at least 1, at most max_inner and the V-cycles left under
// max_v.  Every stop is still decided by a norm of the iterate.
__device__ __forceinline__ int next_inner(const DevState* st, double r, double rmax) {
  const int cap = min(st->max_inner, st->max_v - st->vcycles);
  if (cap <= 1 || !(st->rho > 0.0 && st->rho < 1.0)) return 1;
  const double lr = log(st->rho);
  double need = r > st->tol ? log(st->tol / r) / lr : 0.0;
  if (rmax > st->tol_max) need = fmax(need, log(st->tol_max / rmax) / lr);
  return max(1, min(cap, (int)floor(need + 0.5)));
}

__device__ __forceinline__ unsigned int loop_decision(DevState* st, double r, double rmax, int mode) {
  st->resid = r;
  st->rmax = rmax;
  unsigned int go = 0;
  const bool above = r > st->tol || rmax > st->tol_max;
  if (st->failed == 0) {
    if (mode == 0) {
      st->r0 = r;
      st->vcycles = 0;
      if (!isfinite(r))
        st->failed = 5;  // CHHS_ERR_DIVERGED: a non-finite state or parameter, never "converged"
      else
        go = above ? 1u : 0u;
    } else {
      const int ran = max(st->inner, 1);
      st->vcycles += ran;
      st->checks += 1;
      // contraction per V-cycle over the iteration just finished (kept across
      // steps: the next step's first iteration starts from it)
      if (st->rprev > 0.0 && r > 0.0 && isfinite(r))
        st->rho = fmin(fmax(pow(r / st->rprev, 1.0 / ran), 1e-3), 0.9);
      bool finite = isfinite(r);
      if (!finite || r > 1e8 * (st->r0 + 1.0)) {
        st->failed = 5;  // CHHS_ERR_DIVERGED
      } else if (above) {
        if (st->vcycles >= st->max_v) st->failed = 4;  // CHHS_ERR_NOT_CONVERGED
        else go = 1u;
      }
    }
  }
  st->rprev = r;
  st->inner = go ? next_inner(st, r, rmax) : 1;
  for (int q = 0; q < kMaxInner - 1; ++q) st->go_more[q] = go && st->inner >= 2 + q ? 1 : 0;
  st->go = (int)go;
  return go;
}

// Largest of the three rows' residuals at a cell (the pointwise guard).
__device__ __forceinline__ double row_max(double r1, double r2, double r3s) {
  return fmax(fmax(fabs(r1), fabs(r2)), fabs(r3s));
}

// Block maximum of v (v >= 0); thread 0 returns it.
__device__ __forceinline__ double block_max(double v) {
  __shared__ double shm[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, shm[w]);
  __syncthreads();
  return v;
}

// The norm kernels' last block: the partials (sum of squares, sum of p,
// largest pointwise residual per block) in a fixed order, then the decision.
__device__ __forceinline__ void norm_finish(const double* partials, int nparts, int ncell, DevState* st,
                                            cudaGraphConditionalHandle cond, int mode, int use_cond) {
  double tot[2] = {0.0, 0.0};
  double mx = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    tot[0] += __ldcg(partials + 3 * b);
    tot[1] += __ldcg(partials + 3 * b + 1);
    mx = fmax(mx, __ldcg(partials + 3 * b + 2));
  }
  block_sum<2>(tot);
  mx = block_max(mx);
  if (threadIdx.x != 0) return;
  st->ticket = 0;
  st->pmean = tot[1] / ncell;
  unsigned int go = loop_decision(st, sqrt(tot[0] / ncell), mx, mode);
  if (use_cond) {
    cudaGraphSetConditional(cond, go);
    for (int q = 0; q < st->use_if; ++q) cudaGraphSetConditional(st->cond_if[q], st->inner >= 2 + q ? 1u : 0u);
  }
}

// Blocks per SM of the norm kernels; their threads loop over cells with the
// grid's stride, which amortises the double-precision block sums, and every SM
// holds the same number of blocks.
constexpr int kNormBlocksPerSM = 2;

// Stopping norm sqrt(mean over cells of r_phi^2 + r_mu^2 + (s r_p)^2) on the
// finest grid, in one launch: every block writes its partial sums, and the
// last block to finish (ticket counter) adds the partials in a fixed order and
// takes the loop decision, setting the while-loop condition of the step graph.
// It also records the mean of p (removed when the step is accepted).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_norm(Level<T> L, Coefs<T> K, double* partials, DevState* st,
                                                 cudaGraphConditionalHandle cond, int mode, int use_cond) {
  pdl_enter();
  __shared__ bool last;
  double acc[2] = {0.0, 0.0};
  double mx = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell; c += stride) {
    int i, j, k;
    cell_ijk(c, L.nx, L.ny, i, j, k);
    T n1, n2, n3;
    eval_N<T, DIM, false>(L, K, L.phi, L.mu, L.p, c, i, j, k, n1, n2, n3);
    double r1 = double(L.fphi[c] - n1), r2 = double(L.fmu[c] - n2);
    double r3 = double(K.s) * double(L.fp[c] - n3);
    acc[0] = fma(r1, r1, acc[0]);
    acc[0] = fma(r2, r2, acc[0]);
    acc[0] = fma(r3, r3, acc[0]);
    acc[1] += double(L.p[c]);
    mx = fmax(mx, row_max(r1, r2, r3));
  }
  block_sum<2>(acc);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = acc[0];
    partials[3 * blockIdx.x + 1] = acc[1];
    partials[3 * blockIdx.x + 2] = mx;
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  norm_finish(partials, gridDim.x, L.ncell, st, cond, mode, use_cond);
}

// ---------------------------------------------------------------- mixed precision
//
// Defect correction (iterative refinement): with u the double-precision
// iterate on the finest grid, r = f - N(u) is formed in double; the
// correction e solves N(u + e) - N(u) = r, which single-precision FAS
// V-cycles approximate in correction form (base phi_b = u's phi rounded to
// single); then u <- u + e in double.  Every rounding error of the inner
// solve is relative to the correction, not to u, so the outer loop reaches
// the double-precision tolerance.

// The single-precision finest level of a step: phi^m and phi* rounded, its
// coefficients, and the restriction to the next single-precision level.
template <int DIM>
__device__ __forceinline__ void coef_restrict_f32_body(int bx, Level<double> F, Level<float> G, Coefs<float> K,
                                                              Level<float> Gn, int has_next) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= F.ncell) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  auto ps = [&](int e) { return (float)F.phis[e]; };
  auto pm = [&](int e) { return (float)F.phim[e]; };
  G.phim[c] = pm(c);
  G.phis[c] = ps(c);
  coef_at<float, DIM>(G, K, c, i, j, k, ps, pm(c));
  if (has_next && !(i & 1) && !(j & 1) && (DIM == 2 || !(k & 1)))
    restrict_coef_at<float, double, DIM>(F, Gn, i, j, k, pm, ps);
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_coef_restrict_f32(Level<double> F, Level<float> G, Coefs<float> K,
                                                              Level<float> Gn, int has_next) {
  pdl_enter();
  coef_restrict_f32_body<DIM>(blockIdx.x, F, G, K, Gn, has_next);
}

// The stopping norm of the double-precision iterate, as k_norm, and the
// right-hand side of the next inner solve: f32 = r cut to single precision,
// e = 0, phi_b = phi cut to single precision.
template <int DIM>
__device__ __forceinline__ bool norm_mixed_body(int bx, int nbx, const Level<double>& L, const Coefs<double>& K,
                                                const Level<float>& G,
                                                       double* partials, DevState* st,
                                                       cudaGraphConditionalHandle cond, int mode, int use_cond) {
  __shared__ bool last;
  double acc[2] = {0.0, 0.0};
  double mx = 0.0;
  const int stride = nbx * blockDim.x;
  for (int c = bx * blockDim.x + threadIdx.x; c < L.ncell; c += stride) {
    int i, j, k;
    cell_ijk(c, L.nx, L.ny, i, j, k);
    double n1, n2, n3;
    eval_N<double, DIM, false>(L, K, L.phi, L.mu, L.p, c, i, j, k, n1, n2, n3);
    double r1 = L.fphi[c] - n1, r2 = L.fmu[c] - n2, r3 = L.fp[c] - n3;
    double r3s = K.s * r3;
    acc[0] = fma(r1, r1, acc[0]);
    acc[0] = fma(r2, r2, acc[0]);
    acc[0] = fma(r3s, r3s, acc[0]);
    acc[1] += L.p[c];
    mx = fmax(mx, row_max(r1, r2, r3s));
    G.fphi[c] = f64_to_f32_rz(r1);
    G.fmu[c] = f64_to_f32_rz(r2);
    G.fp[c] = f64_to_f32_rz(r3);
    G.phi[c] = 0.f;
    G.mu[c] = 0.f;
    G.p[c] = 0.f;
    G.phib[c] = f64_to_f32_rz(L.phi[c]);
  }
  block_sum<2>(acc);
  mx = block_max(mx);
  if (threadIdx.x == 0) {
    partials[3 * bx] = acc[0];
    partials[3 * bx + 1] = acc[1];
    partials[3 * bx + 2] = mx;
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == nbx - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  norm_finish(partials, nbx, L.ncell, st, cond, mode, use_cond);
  return true;
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_norm_mixed(const __grid_constant__ Level<double> L, Coefs<double> K,
                                                       const __grid_constant__ Level<float> G,
                                                       double* partials, DevState* st,
                                                       cudaGraphConditionalHandle cond, int mode, int use_cond) {
  pdl_enter();
  norm_mixed_body<DIM>(blockIdx.x, gridDim.x, L, K, G, partials, st, cond, mode, use_cond);
}

// u <- u + e in double precision.
static __device__ __forceinline__ void mixed_update_body(int bx, Level<double> L, Level<float> G) {
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= L.ncell) return;
  L.phi[c] += (double)G.phi[c];
  L.mu[c] += (double)G.mu[c];
  L.p[c] += (double)G.p[c];
}

static __global__ void __launch_bounds__(kBlock) k_mixed_update(Level<double> L, Level<float> G) {
  pdl_enter();
  mixed_update_body(blockIdx.x, L, G);
}

// ---------------------------------------------------------------- step frame

// phi* = 3/2 phi^m - 1/2 phi^{m-1} (Eq. 2.4); f_phi = phi^m;
// f_mu = -phi* - (1/4) eps^2 Lap_h phi^{m-1}, carried shifted by (phi^m)^3/4
// as the plain form's N2 is (cubic_P); f_p = 0; initial guess
// phi = 2 phi^m - phi^{m-1} (mu and p keep the previous step's values).
// Fused: the finest level's coefficients (phi* of the neighbours formed on
// the fly) and the restriction of phi^m, phi* to the next level (has_next).
template <int DIM>
__device__ __forceinline__ void setup_coef_body(int bx, Level<double> L, const double* phimm1, double eps2,
                                                       const DevState* st, Coefs<double> K, Level<double> Cn,
                                                       int has_next) {
  if (st->failed) return;
  int c = bx * blockDim.x + threadIdx.x;
  if (c >= L.ncell) return;
  int i, j, k;
  cell_ijk(c, L.nx, L.ny, i, j, k);
  double pm = L.phim[c], pmm = phimm1[c];
  double lap = 0.0;
  const int sy = L.nx, sz = L.nx * L.ny;
  if (i > 0) lap += phimm1[c - 1] - pmm;
  if (i + 1 < L.nx) lap += phimm1[c + 1] - pmm;
  if (j > 0) lap += phimm1[c - sy] - pmm;
  if (j + 1 < L.ny) lap += phimm1[c + sy] - pmm;
  if (DIM == 3) {
    if (k > 0) lap += phimm1[c - sz] - pmm;
    if (k + 1 < L.nz) lap += phimm1[c + sz] - pmm;
  }
  double ps = 1.5 * pm - 0.5 * pmm;
  L.phis[c] = ps;
  L.fphi[c] = pm;
  L.fmu[c] = (-ps - 0.25 * eps2 * L.ih2 * lap) + 0.25 * pm * pm * pm;
  L.fp[c] = 0.0;
  L.phi[c] = 2.0 * pm - pmm;
  auto psf = [&](int e) { return 1.5 * L.phim[e] - 0.5 * phimm1[e]; };
  auto pmf = [&](int e) { return L.phim[e]; };
  coef_at<double, DIM>(L, K, c, i, j, k, psf, pm);
  if (has_next && !(i & 1) && !(j & 1) && (DIM == 2 || !(k & 1)))
    restrict_coef_at<double, double, DIM>(L, Cn, i, j, k, pmf, psf);
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_setup_coef(Level<double> L, const double* phimm1, double eps2,
                                                       const DevState* st, Coefs<double> K, Level<double> Cn,
                                                       int has_next) {
  pdl_enter();
  setup_coef_body<DIM>(blockIdx.x, L, phimm1, eps2, st, K, Cn, has_next);
}

// Accept the step: phi^{m-1} <- phi^m, phi^m <- phi^{m+1}, p <- p - mean(p).
static __device__ __forceinline__ void advance_body(int bx, Level<double> L, double* phimm1, DevState* st) {
  if (st->failed) return;
  int c = bx * blockDim.x + threadIdx.x;
  if (c == 0) {
    st->steps_done += 1;
    st->vtotal += st->vcycles;
  }
  if (c >= L.ncell) return;
  phimm1[c] = L.phim[c];
  L.phim[c] = L.phi[c];
  L.p[c] -= st->pmean;
}

static __global__ void __launch_bounds__(kBlock) k_advance(Level<double> L, double* phimm1, DevState* st) {
  pdl_enter();
  advance_body(blockIdx.x, L, phimm1, st);
}

// ---------------------------------------------------------------- coarse tail

// The bottom of a V-cycle -- from some level down to the coarsest and back --
// run by a single block.  On these small levels a kernel launch costs more
// than the work, so the whole tail is one launch with block barriers between
// passes.  Global memory written by the block is visible to it after
// __syncthreads.
template <typename T>
struct Tail {
  Level<T> lev[kTailMaxLevels];
  int n;        // levels in the tail; the last one is the coarsest
  int nu1, nu2;
  int top_rhs;  // complete the FAS right-hand side of the tail's top level first
  int coarsest_f64;  // single-precision correction form: solve the coarsest grid in double precision
};

// Groups of three warps in the tail block for the split update (warp 15 idles).
constexpr int kTailGroups = kTailThreads / 96;

template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void tail_smooth(const Level<T>& L, const Coefs<T>& K, int colour, bool rhs) {
  const int hw = (L.nx + 1) >> 1;
  const int total = hw * L.ny * L.nz;
  if constexpr (!CORR && sizeof(T) == 8) {
    // plain double precision: split update, groups of three warps, named
    // barrier per group; every group runs the same number of rounds
    __shared__ float xch[2][kTailGroups][4 * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp / 3, role = warp - 3 * g;
    if (g < kTailGroups) {
      const int rounds = (total + 32 * kTailGroups - 1) / (32 * kTailGroups);
      for (int r = 0; r < rounds; ++r) {
        const int t = r * 32 * kTailGroups + g * 32 + lane;
        const int row = small_div(t, L.rhw);
        const int ti = t - row * hw;
        const int k = small_div(row, L.rny);
        const int j = row - k * L.ny;
        const int i = 2 * ti + ((j + k + colour) & 1);
        const bool act = t < total && i < L.nx;
        const int c = act ? i + L.nx * (j + L.ny * k) : 0;
        cell_update_split<DIM>(L, K, role, act, c, i, j, k, rhs, &xch[r & 1][g][lane], [g] {
          asm volatile("bar.sync %0, 96;" ::"r"(g + 1) : "memory");
        });
      }
    }
  } else {
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int row = small_div(t, L.rhw);
      const int ti = t - row * hw;
      const int k = small_div(row, L.rny);
      const int j = row - k * L.ny;
      const int i = 2 * ti + ((j + k + colour) & 1);
      if (i >= L.nx) continue;
      const int c = i + L.nx * (j + L.ny * k);
      T f1, f2, f3;
      cell_rhs<T, DIM, CORR>(L, K, c, i, j, k, rhs, f1, f2, f3);
      cell_update<T, DIM, CORR>(L, K, c, i, j, k, f1, f2, f3);
    }
  }
  __syncthreads();
}

template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void tail_rhs(const Level<T>& L, const Coefs<T>& K) {
  if constexpr (!CORR && sizeof(T) == 8) {
    // plain double precision: the three rows of N(R u) on three warps of a group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp / 3, role = warp - 3 * g;
    if (g < kTailGroups)
      for (int c = g * 32 + lane; c < L.ncell; c += 32 * kTailGroups) {
        int i, j, k;
        cell_ijk_small(c, L, i, j, k);
        double u;
        f_row(L, role)[c] += n_row<DIM>(L, K, role, L.phi0, L.mu0, L.p0, c, i, j, k, u);
      }
  } else {
    for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
      int i, j, k;
      cell_ijk_small(c, L, i, j, k);
      T f1, f2, f3;
      cell_rhs<T, DIM, CORR>(L, K, c, i, j, k, true, f1, f2, f3);
    }
  }
  __syncthreads();
}

// Residual and restriction inside the tail: one thread per fine cell, the
// 2^d children of a coarse cell in adjacent lanes (child d = t mod 2^d), their
// values summed by shuffles in a fixed order.  Every thread of the block
// takes part in the shuffles (the round count is uniform).
template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void tail_restrict(const Level<T>& F, const Level<T>& C, const Coefs<T>& K) {
  constexpr int NCH = DIM == 3 ? 8 : 4;
  if constexpr (!CORR && sizeof(T) == 8) {
    // plain double precision: the phi, pressure and mu rows on the three warps
    // of a group (n_row), each writing its own coarse values
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp / 3, role = warp - 3 * g;
    if (g < kTailGroups) {
      const double w = DIM == 3 ? 0.125 : 0.25;
      const int total = C.ncell * NCH;
      const int rounds = (total + 32 * kTailGroups - 1) / (32 * kTailGroups);
      for (int r = 0; r < rounds; ++r) {
        const int t = r * 32 * kTailGroups + g * 32 + lane;
        const bool act = t < total;
        const int q = t / NCH, d = t % NCH;
        double rr = 0.0, u = 0.0;
        if (act) {
          int I, J, KK;
          cell_ijk_small(q, C, I, J, KK);
          const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * KK + (d >> 2);
          const int c = i + F.nx * (j + F.ny * k);
          const double n = n_row<DIM>(F, K, role, F.phi, F.mu, F.p, c, i, j, k, u);
          rr = f_row(F, role)[c] - n;
        }
#pragma unroll
        for (int o = 1; o < NCH; o <<= 1) {
          rr += __shfl_xor_sync(0xffffffffu, rr, o);
          u += __shfl_xor_sync(0xffffffffu, u, o);
        }
        if (act && d == 0) {
          if (role == 0) {
            C.fphi[q] = w * rr;
            C.phi[q] = C.phi0[q] = w * u;
          } else if (role == 1) {
            C.fp[q] = w * rr;
            C.p[q] = C.p0[q] = w * u;
          } else {
            C.fmu[q] = w * rr;
            C.mu[q] = C.mu0[q] = w * u;
          }
        }
      }
    }
    __syncthreads();
    return;
  }
  constexpr int NV = CORR ? 7 : 6;
  const T w = DIM == 3 ? T(0.125) : T(0.25);
  const int total = C.ncell * NCH;
  const int rounds = (total + (int)blockDim.x - 1) / (int)blockDim.x;
  for (int r = 0; r < rounds; ++r) {
    const int t = r * (int)blockDim.x + (int)threadIdx.x;
    const bool act = t < total;
    const int q = t / NCH, d = t % NCH;
    T v[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) v[m] = T(0);
    if (act) {
      int I, J, KK;
      cell_ijk_small(q, C, I, J, KK);
      const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * KK + (d >> 2);
      const int c = i + F.nx * (j + F.ny * k);
      T n1, n2, n3;
      eval_N<T, DIM, CORR>(F, K, F.phi, F.mu, F.p, c, i, j, k, n1, n2, n3);
      v[0] = F.fphi[c] - n1;
      v[1] = F.fmu[c] - n2;
      v[2] = F.fp[c] - n3;
      v[3] = F.phi[c];
      v[4] = F.mu[c];
      v[5] = F.p[c];
      if (CORR) v[NV - 1] = F.phib[c];
    }
#pragma unroll
    for (int o = 1; o < NCH; o <<= 1)
#pragma unroll
      for (int m = 0; m < NV; ++m) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
    if (act && d == 0) {
      C.fphi[q] = w * v[0];
      C.fmu[q] = w * v[1];
      C.fp[q] = w * v[2];
      C.phi[q] = C.phi0[q] = w * v[3];
      C.mu[q] = C.mu0[q] = w * v[4];
      C.p[q] = C.p0[q] = w * v[5];
      if (CORR) C.phib[q] = w * v[NV - 1];
    }
  }
  __syncthreads();
}

template <typename T, int DIM>
__device__ __forceinline__ void tail_prolong(const Level<T>& F, const Level<T>& C) {
  for (int c = threadIdx.x; c < F.ncell; c += blockDim.x) {
    int i, j, k;
    cell_ijk_small(c, F, i, j, k);
    int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (DIM == 3 ? (k >> 1) : 0));
    F.phi[c] += C.phi[q] - C.phi0[q];
    F.mu[c] += C.mu[q] - C.mu0[q];
    F.p[c] += C.p[q] - C.p0[q];
  }
  __syncthreads();
}

// The coarsest grid: red-black sweeps until the residual norm has fallen by
// 1e-2 (the coarsest grids here have a handful of cells and a nearly
// diagonal operator, and a coarse-grid correction inside a V-cycle that
// contracts by ~0.1 needs no more; a tighter target was measured to leave
// the V-cycle count unchanged), or, after the first 8 sweeps, stops falling
// (the floor; early sweeps of this coupled system may raise the residual
// before it falls), or after 2000 sweeps.  A slowly contracting solve (a
// large coarsest grid) keeps sweeping.  The norm only decides when to stop,
// so it is summed in single precision, over the warps that hold cells, and
// compared squared (no square root or division).
constexpr int kCoarsestMaxSweeps = 2000;
constexpr float kCoarsestTarget2 = 1e-4f;  // (1e-2)^2

template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void coarsest_solve(const Level<T>& L, const Coefs<T>& K) {
  __shared__ float sh_part[kTailThreads / 32];
  const int nw = min((L.ncell + 31) >> 5, (int)(blockDim.x >> 5));
  float acc0 = -1.f, prev = 0.f;
  for (int it = 0; it <= kCoarsestMaxSweeps; ++it) {
    // every warp writes its partial (zero without cells)
    T acc = T(0);
    if constexpr (!CORR && sizeof(T) == 8) {
      // plain double precision: the three rows on the three warps of a group
      const int warp = threadIdx.x >> 5, g = warp / 3, role = warp - 3 * g;
      if (g < kTailGroups)
        for (int c = g * 32 + (threadIdx.x & 31); c < L.ncell; c += 32 * kTailGroups) {
          int i, j, k;
          cell_ijk_small(c, L, i, j, k);
          double u;
          double r = f_row(L, role)[c] - n_row<DIM>(L, K, role, L.phi, L.mu, L.p, c, i, j, k, u);
          if (role == 1) r *= K.s;
          acc += r * r;
        }
    } else {
      if ((int)threadIdx.x < nw * 32)
        for (int c = threadIdx.x; c < L.ncell; c += nw * 32) {
          int i, j, k;
          cell_ijk_small(c, L, i, j, k);
          T n1, n2, n3;
          eval_N<T, DIM, CORR>(L, K, L.phi, L.mu, L.p, c, i, j, k, n1, n2, n3);
          T r1 = L.fphi[c] - n1, r2 = L.fmu[c] - n2, r3 = K.s * (L.fp[c] - n3);
          acc += r1 * r1 + r2 * r2 + r3 * r3;
        }
    }
    const float a = warp_sum((float)acc);
    if ((threadIdx.x & 31) == 0) sh_part[threadIdx.x >> 5] = a;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh_part[w];
    if (acc0 < 0.f) acc0 = tot;
    if (!(tot > kCoarsestTarget2 * acc0) || tot < 1e-37f) break;
    if (it >= 8 && tot >= prev) break;
    prev = tot;
    // the passes end in __syncthreads, so sh_part is read by all before it is rewritten
    for (int colour = 0; colour < 2; ++colour) tail_smooth<T, DIM, CORR>(L, K, colour, false);
  }
  __syncthreads();
}

// Fields of a tail level held in shared memory, in carving order.  The
// per-step coefficients (phi^m, a, M, their sums, the smoother's constants) are copied in
// on every level, the state and right-hand sides (phi, mu, p, f, R u, phi_b)
// only on the tail's top level; the levels below are computed in place.
template <int DIM, bool CORR>
__host__ __device__ constexpr int tail_fields() { return 22 + (DIM == 3 ? 2 : 0) + (CORR ? 1 : 0); }

__host__ __device__ inline size_t tail_align(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int DIM, bool CORR>
__host__ __device__ inline size_t tail_smem_bytes(const int* ncell, int n, int coarsest_f64 = 0) {
  size_t b = 0;
  for (int l = 0; l < n; ++l) b += tail_fields<DIM, CORR>() * tail_align(sizeof(T) * ncell[l]);
  // the double-precision copy of the coarsest grid (coarsest_solve_f64)
  if (coarsest_f64 && n > 0) b += tail_fields<DIM, CORR>() * tail_align(sizeof(double) * ncell[n - 1]);
  return b;
}

// Level l of the tail with its arrays in shared memory.  Every thread forms
// the pointers itself from the shared-memory base, so the compiler sees
// shared-memory accesses (no level table in memory, no generic loads).
template <typename T, int DIM, bool CORR>
__device__ __forceinline__ Level<T> tail_level(const Tail<T>& tl, int l, unsigned char* smem) {
  size_t off = 0;
  for (int q = 0; q < l; ++q) off += tail_fields<DIM, CORR>() * tail_align(sizeof(T) * tl.lev[q].ncell);
  Level<T> L = tl.lev[l];
  const size_t st = tail_align(sizeof(T) * L.ncell);
  int q = 0;
  auto carve = [&]() { return reinterpret_cast<T*>(smem + off + (q++) * st); };
  L.phi = carve(); L.mu = carve(); L.p = carve();
  L.fphi = carve(); L.fmu = carve(); L.fp = carve();
  L.phim = carve(); L.phi0 = carve(); L.mu0 = carve(); L.p0 = carve();
  L.ax = carve(); L.ay = carve(); L.Mx = carve(); L.My = carve();
  L.sM = carve(); L.sa = carve();
  L.cAe = carve(); L.cC = carve(); L.cGn = carve(); L.cHn = carve(); L.cQ = carve(); L.cH = carve();
  if (DIM == 3) { L.az = carve(); L.Mz = carve(); }
  if (CORR) L.phib = carve();
  L.phis = nullptr;
  return L;
}

// The coarsest solve of a single-precision correction-form V-cycle carried
// out in double precision: the coarsest grid's fields are widened into a
// double-precision copy (its per-step coefficients, computed in single
// precision, are widened exactly), the sweeps and the stopping test of
// coarsest_solve run on the copy, and the correction is rounded back.
template <int DIM>
__device__ __forceinline__ void coarsest_solve_f64(const Level<float>& S, const Coefs<float>& K,
                                                   unsigned char* smem) {
  Level<double> D;
  D.nx = S.nx; D.ny = S.ny; D.nz = S.nz; D.ncell = S.ncell;
  D.rnx = S.rnx; D.rny = S.rny; D.rhw = S.rhw;
  D.ih2 = S.ih2; D.h2 = S.h2; D.sih2 = S.sih2; D.e34ih2 = S.e34ih2;
  const size_t st = tail_align(sizeof(double) * S.ncell);
  int q = 0;
  auto carve = [&]() { return reinterpret_cast<double*>(smem + (q++) * st); };
  const float* src[22] = {S.phi, S.mu, S.p, S.fphi, S.fmu, S.fp, S.phim, S.phib, S.ax, S.ay, S.Mx, S.My,
                          S.sM, S.sa, S.cAe, S.cC, S.cGn, S.cHn, S.cQ, S.cH, S.az, S.Mz};
  D.phi = carve(); D.mu = carve(); D.p = carve(); D.fphi = carve(); D.fmu = carve(); D.fp = carve();
  D.phim = carve(); D.phib = carve(); D.ax = carve(); D.ay = carve(); D.Mx = carve(); D.My = carve();
  D.sM = carve(); D.sa = carve(); D.cAe = carve(); D.cC = carve(); D.cGn = carve(); D.cHn = carve();
  D.cQ = carve(); D.cH = carve();
  D.az = DIM == 3 ? carve() : nullptr;
  D.Mz = DIM == 3 ? carve() : nullptr;
  D.phis = D.phi0 = D.mu0 = D.p0 = nullptr;
  double* dst[22] = {D.phi, D.mu, D.p, D.fphi, D.fmu, D.fp, D.phim, D.phib, D.ax, D.ay, D.Mx, D.My,
                     D.sM, D.sa, D.cAe, D.cC, D.cGn, D.cHn, D.cQ, D.cH, D.az, D.Mz};
  const int nf = DIM == 3 ? 22 : 20;
  for (int f = 0; f < nf; ++f)
    for (int c = threadIdx.x; c < S.ncell; c += blockDim.x) dst[f][c] = (double)src[f][c];
  __syncthreads();
  const Coefs<double> KD{(double)K.s, (double)K.gamma, (double)K.e34};
  coarsest_solve<double, DIM, true>(D, KD);
  for (int c = threadIdx.x; c < S.ncell; c += blockDim.x) {
    S.phi[c] = (float)D.phi[c];
    S.mu[c] = (float)D.mu[c];
    S.p[c] = (float)D.p[c];
  }
  __syncthreads();
}

template <typename T, int DIM, bool CORR>
__device__ __forceinline__ void tail_body(const Tail<T>& tl, const Coefs<T>& K) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  const int n = tl.n;
  // Copy in: per cell, every field is loaded before any is stored, so a
  // thread's loads are all in flight together.
  for (int l = 0; l < n; ++l) {
    const Level<T>& G = tl.lev[l];
    const Level<T> S = tail_level<T, DIM, CORR>(tl, l, tail_smem);
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
      T v[15];
      v[0] = G.phim[c]; v[1] = G.ax[c]; v[2] = G.ay[c]; v[3] = G.Mx[c]; v[4] = G.My[c];
      v[5] = G.sM[c]; v[6] = G.sa[c]; v[7] = G.cAe[c]; v[8] = G.cC[c]; v[9] = G.cGn[c];
      v[10] = G.cHn[c]; v[11] = G.cQ[c]; v[14] = G.cH[c];
      if (DIM == 3) { v[12] = G.az[c]; v[13] = G.Mz[c]; }
      S.phim[c] = v[0]; S.ax[c] = v[1]; S.ay[c] = v[2]; S.Mx[c] = v[3]; S.My[c] = v[4];
      S.sM[c] = v[5]; S.sa[c] = v[6]; S.cAe[c] = v[7]; S.cC[c] = v[8]; S.cGn[c] = v[9];
      S.cHn[c] = v[10]; S.cQ[c] = v[11]; S.cH[c] = v[14];
      if (DIM == 3) { S.az[c] = v[12]; S.Mz[c] = v[13]; }
      if (l == 0) {
        T u[10];
        u[0] = G.phi[c]; u[1] = G.mu[c]; u[2] = G.p[c]; u[3] = G.fphi[c]; u[4] = G.fmu[c]; u[5] = G.fp[c];
        u[6] = G.phi0[c]; u[7] = G.mu0[c]; u[8] = G.p0[c];
        if (CORR) u[9] = G.phib[c];
        S.phi[c] = u[0]; S.mu[c] = u[1]; S.p[c] = u[2]; S.fphi[c] = u[3]; S.fmu[c] = u[4]; S.fp[c] = u[5];
        S.phi0[c] = u[6]; S.mu0[c] = u[7]; S.p0[c] = u[8];
        if (CORR) S.phib[c] = u[9];
      }
    }
  }
  __syncthreads();
  auto copy = [&](T* dst, const T* src, int nc) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) dst[c] = src[c];
  };

  for (int l = 0; l + 1 < n; ++l) {
    const Level<T> L = tail_level<T, DIM, CORR>(tl, l, tail_smem);
    bool rhs = l > 0 || tl.top_rhs;
    if (rhs && tl.nu1 == 0) {
      tail_rhs<T, DIM, CORR>(L, K);
      rhs = false;
    }
    for (int it = 0; it < tl.nu1; ++it)
      for (int colour = 0; colour < 2; ++colour) tail_smooth<T, DIM, CORR>(L, K, colour, rhs && it == 0);
    tail_restrict<T, DIM, CORR>(L, tail_level<T, DIM, CORR>(tl, l + 1, tail_smem), K);
  }
  {
    const Level<T> Lc = tail_level<T, DIM, CORR>(tl, n - 1, tail_smem);
    if (n > 1 || tl.top_rhs) tail_rhs<T, DIM, CORR>(Lc, K);
    if constexpr (sizeof(T) == 4 && CORR) {
      if (tl.coarsest_f64) {
        size_t off = 0;
        for (int q = 0; q < n; ++q) off += tail_fields<DIM, CORR>() * tail_align(sizeof(T) * tl.lev[q].ncell);
        coarsest_solve_f64<DIM>(Lc, K, tail_smem + off);
      } else {
        coarsest_solve<T, DIM, CORR>(Lc, K);
      }
    } else {
      coarsest_solve<T, DIM, CORR>(Lc, K);
    }
  }
  for (int l = n - 2; l >= 0; --l) {
    const Level<T> L = tail_level<T, DIM, CORR>(tl, l, tail_smem);
    tail_prolong<T, DIM>(L, tail_level<T, DIM, CORR>(tl, l + 1, tail_smem));
    for (int it = 0; it < tl.nu2; ++it)
      for (int colour = 0; colour < 2; ++colour) tail_smooth<T, DIM, CORR>(L, K, colour, false);
  }

  const Level<T>& G = tl.lev[0];
  const Level<T> S = tail_level<T, DIM, CORR>(tl, 0, tail_smem);
  copy(G.phi, S.phi, G.ncell);
  copy(G.mu, S.mu, G.ncell);
  copy(G.p, S.p, G.ncell);
}

template <typename T, int DIM, bool CORR>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const __grid_constant__ Tail<T> tl, Coefs<T> K) {
  pdl_enter();
  tail_body<T, DIM, CORR>(tl, K);
}

// ---------------------------------------------------------------- diagnostics

// Per block: sum phi, sum phi^4, sum phi^2, sum over interior faces of
// (D phi)^2, sum (phi - psi)^2, sum over interior faces of (D(phi - psi))^2.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_energy_partial(const double* phi, const double* psi, int nx,
                                                           int ny, int nz, double ih, double* partials) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int n = nx * ny * nz;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (c < n) {
    int i, j, k;
    cell_ijk(c, nx, ny, i, j, k);
    double f = phi[c], d = f - psi[c];
    v[0] = f;
    v[1] = f * f * f * f;
    v[2] = f * f;
    v[4] = d * d;
    const int sy = nx, sz = nx * ny;
    auto face = [&](int e) {
      double g = (phi[e] - f) * ih;
      double gd = ((phi[e] - psi[e]) - d) * ih;
      v[3] += g * g;
      v[5] += gd * gd;
    };
    if (i + 1 < nx) face(c + 1);
    if (j + 1 < ny) face(c + sy);
    if (DIM == 3 && k + 1 < nz) face(c + sz);
  }
  block_sum<6>(v);
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) partials[blockIdx.x * 6 + q] = v[q];
}

// Dissipation terms of the last solved step (Eq. 2.23 and its proof):
// per block the sums over interior faces of (D mu)^2 and u^2 with
// u = -D p - gamma (A phi*) D mu (Eq. 2.3; u = 0 on boundary faces), and the
// largest |div_h u| over the block's cells.  mu, p, phi* are the handle's.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_dissip_partial(Level<double> L, double gamma, double ih,
                                                           double* partials) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  double dmax = 0.0;
  if (c < L.ncell) {
    int i, j, k;
    cell_ijk(c, L.nx, L.ny, i, j, k);
    const double muc = L.mu[c], pc = L.p[c], psc = L.phis[c];
    double div = 0.0;
    auto face = [&](int e, bool plus) {
      double gmu = (L.mu[e] - muc) * ih;   // D mu, outward from c
      double u = -(L.p[e] - pc) * ih - gamma * 0.5 * (psc + L.phis[e]) * gmu;
      div += u * ih;
      if (plus) {  // each interior face counted once, from its lower cell
        v[0] += gmu * gmu;
        v[1] += u * u;
      }
    };
    const int sy = L.nx, sz = L.nx * L.ny;
    if (i > 0) face(c - 1, false);
    if (i + 1 < L.nx) face(c + 1, true);
    if (j > 0) face(c - sy, false);
    if (j + 1 < L.ny) face(c + sy, true);
    if (DIM == 3) {
      if (k > 0) face(c - sz, false);
      if (k + 1 < L.nz) face(c + sz, true);
    }
    dmax = fabs(div);
  }
  block_sum<2>(v);
  __shared__ double shm[32];
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) dmax = fmax(dmax, shm[w]);
    partials[3 * blockIdx.x] = v[0];
    partials[3 * blockIdx.x + 1] = v[1];
    partials[3 * blockIdx.x + 2] = dmax;
  }
}

// The velocity of Eq. 2.3 on the face grid: ux[c] (uy, uz) is the
// component on the face between cell c and its +x (+y, +z) neighbour, zero on
// boundary faces; the same face formula as k_dissip_partial.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_velocity(Level<double> L, double gamma, double ih, double* ux,
                                                     double* uy, double* uz) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.ncell) return;
  int i, j, k;
  cell_ijk(c, L.nx, L.ny, i, j, k);
  const double muc = L.mu[c], pc = L.p[c], psc = L.phis[c];
  auto face = [&](bool in, int e) {
    if (!in) return 0.0;
    const double gmu = (L.mu[e] - muc) * ih;
    return -(L.p[e] - pc) * ih - gamma * 0.5 * (psc + L.phis[e]) * gmu;
  };
  ux[c] = face(i + 1 < L.nx, c + 1);
  uy[c] = face(j + 1 < L.ny, c + L.nx);
  if (DIM == 3) uz[c] = face(k + 1 < L.nz, c + L.nx * L.ny);
}

static __global__ void k_dissip_finish(const double* partials, int nparts, DevState* st) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0, m = 0.0;
  for (int q = 0; q < nparts; ++q) {
    a += partials[3 * q];
    b += partials[3 * q + 1];
    m = fmax(m, partials[3 * q + 2]);
  }
  st->diag[0] = a;
  st->diag[1] = b;
  st->diag[2] = m;
}

static __global__ void k_energy_finish(const double* partials, int nparts, DevState* st) {
  double tot[6];
  sum_partials<6>(partials, nparts, tot);
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) st->diag[q] = tot[q];
}

}  // namespace chhs_dev
