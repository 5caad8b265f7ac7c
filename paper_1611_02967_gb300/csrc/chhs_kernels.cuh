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
// Grid functions are stored x fastest, interior cells only.  The homogeneous
// Neumann ghosts of Appendix A (ghost = mirror of its neighbour) make every
// boundary-face difference vanish, so boundary faces carry no flux and the
// stencil loops below simply skip them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace chhs_dev {

constexpr int kBlock = 256;

template <typename T>
struct Level {
  T *phi, *mu, *p;     // unknowns
  T *fphi, *fmu, *fp;  // right-hand sides
  T *phim, *phis;      // phi^m and phi* restricted to this level (fixed in a step)
  T *phi0, *mu0, *p0;  // restricted iterate R u kept for the FAS correction
  int nx, ny, nz;      // nz == 1 in 2D
  int ncell;
  T ih2;               // 1 / h^2 on this level
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
  double resid;    // last fine-grid stopping norm
  double r0;       // stopping norm at the start of the step
  double pmean;    // mean of p, removed when the step is accepted
  double diag[8];  // reduction results (mass, energies)
};

// chi(a, b) = (a^2 + b^2)(a + b) / 4 (Eq. 2.4) and d chi / d a.
template <typename T>
__device__ __forceinline__ T chi(T a, T b) { return T(0.25) * (a * a + b * b) * (a + b); }
template <typename T>
__device__ __forceinline__ T dchi_da(T a, T b) { return T(0.25) * (T(3) * a * a + T(2) * a * b + b * b); }

__device__ __forceinline__ void cell_ijk(int c, int nx, int ny, int& i, int& j, int& k) {
  i = c % nx;
  int r = c / nx;
  j = r % ny;
  k = r / ny;
}

// Face sums of one cell: for each interior face f with neighbour e,
//   a_f = A_h phi* = (phi*_c + phi*_e)/2,  M_f = 1 + gamma a_f^2.
template <typename T>
struct Sums {
  T Mdmu, adp, admu, dphi, dp, M, a;
  int m;  // number of interior faces n_c
};

template <typename T, int DIM>
__device__ __forceinline__ void face_sums(const Level<T>& L, const Coefs<T>& K, int c, int i, int j,
                                          int k, T phic, T muc, T pc, T psc, Sums<T>& S) {
  S.Mdmu = S.adp = S.admu = S.dphi = S.dp = S.M = S.a = T(0);
  S.m = 0;
  auto face = [&](int e) {
    T af = T(0.5) * (psc + L.phis[e]);
    T Mf = T(1) + K.gamma * af * af;
    T dmu = L.mu[e] - muc;
    T dp = L.p[e] - pc;
    S.Mdmu += Mf * dmu;
    S.adp += af * dp;
    S.admu += af * dmu;
    S.dphi += L.phi[e] - phic;
    S.dp += dp;
    S.M += Mf;
    S.a += af;
    S.m += 1;
  };
  const int sy = L.nx, sz = L.nx * L.ny;
  if (i > 0) face(c - 1);
  if (i + 1 < L.nx) face(c + 1);
  if (j > 0) face(c - sy);
  if (j + 1 < L.ny) face(c + sy);
  if (DIM == 3) {
    if (k > 0) face(c - sz);
    if (k + 1 < L.nz) face(c + sz);
  }
}

// N(u) at cell c.
template <typename T, int DIM>
__device__ __forceinline__ void apply_N(const Level<T>& L, const Coefs<T>& K, int c, int i, int j,
                                        int k, T& n1, T& n2, T& n3) {
  T phic = L.phi[c], muc = L.mu[c], pc = L.p[c];
  Sums<T> S;
  face_sums<T, DIM>(L, K, c, i, j, k, phic, muc, pc, L.phis[c], S);
  n1 = phic - K.s * L.ih2 * (S.Mdmu + S.adp);
  n2 = muc - chi(phic, L.phim[c]) + K.e34 * L.ih2 * S.dphi;
  n3 = -L.ih2 * (S.dp + K.gamma * S.admu);
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
//   dphi = (R1 - Ae R2 - (C/Dn) R3) / (1 + Ae B),  dmu = R2 + B dphi,
//   dp = (R3 - G dmu) / Dn.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_smooth(Level<T> L, Coefs<T> K, int colour) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.ncell) return;
  int i, j, k;
  cell_ijk(c, L.nx, L.ny, i, j, k);
  if (((i + j + k) & 1) != colour) return;
  T phic = L.phi[c], muc = L.mu[c], pc = L.p[c], phimc = L.phim[c];
  Sums<T> S;
  face_sums<T, DIM>(L, K, c, i, j, k, phic, muc, pc, L.phis[c], S);
  T n1 = phic - K.s * L.ih2 * (S.Mdmu + S.adp);
  T n2 = muc - chi(phic, phimc) + K.e34 * L.ih2 * S.dphi;
  T n3 = -L.ih2 * (S.dp + K.gamma * S.admu);
  T R1 = L.fphi[c] - n1, R2 = L.fmu[c] - n2, R3 = L.fp[c] - n3;
  T inv_m = T(1) / T(S.m);
  T Ae = K.s * L.ih2 * (S.M - K.gamma * S.a * S.a * inv_m);
  T CD = K.s * S.a * inv_m;
  T G = K.gamma * L.ih2 * S.a;
  T B = dchi_da(phic, phimc) + K.e34 * L.ih2 * T(S.m);
  T dphi = (R1 - Ae * R2 - CD * R3) / (T(1) + Ae * B);
  T dmu = R2 + B * dphi;
  T dp = (R3 - G * dmu) * inv_m / L.ih2;
  L.phi[c] = phic + dphi;
  L.mu[c] = muc + dmu;
  L.p[c] = pc + dp;
}

// ---------------------------------------------------------------- transfers

// For each coarse cell: u_c = R u (mean of the 2^d children), kept twice (as
// the coarse iterate and as u_c^0), and the restricted fine residual R r as
// the first part of the FAS right-hand side.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_residual_restrict(Level<T> F, Level<T> C, Coefs<T> K) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= C.ncell) return;
  int I, J, KK;
  cell_ijk(q, C.nx, C.ny, I, J, KK);
  T sphi = 0, smu = 0, sp = 0, r1 = 0, r2 = 0, r3 = 0;
  const int kz = DIM == 3 ? 2 : 1;
  for (int dk = 0; dk < kz; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int i = 2 * I + di, j = 2 * J + dj, k = 2 * KK + dk;
        int c = i + F.nx * (j + F.ny * k);
        T n1, n2, n3;
        apply_N<T, DIM>(F, K, c, i, j, k, n1, n2, n3);
        r1 += F.fphi[c] - n1;
        r2 += F.fmu[c] - n2;
        r3 += F.fp[c] - n3;
        sphi += F.phi[c];
        smu += F.mu[c];
        sp += F.p[c];
      }
  const T w = DIM == 3 ? T(0.125) : T(0.25);
  C.phi[q] = C.phi0[q] = w * sphi;
  C.mu[q] = C.mu0[q] = w * smu;
  C.p[q] = C.p0[q] = w * sp;
  C.fphi[q] = w * r1;
  C.fmu[q] = w * r2;
  C.fp[q] = w * r3;
}

// f_c += N_c(u_c^0): completes the FAS right-hand side on the coarse grid.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_coarse_rhs(Level<T> C, Coefs<T> K) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= C.ncell) return;
  int i, j, k;
  cell_ijk(q, C.nx, C.ny, i, j, k);
  T n1, n2, n3;
  apply_N<T, DIM>(C, K, q, i, j, k, n1, n2, n3);
  C.fphi[q] += n1;
  C.fmu[q] += n2;
  C.fp[q] += n3;
}

// u += P(u_c - u_c^0), P piecewise constant.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong(Level<T> F, Level<T> C) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= F.ncell) return;
  int i, j, k;
  cell_ijk(c, F.nx, F.ny, i, j, k);
  int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (DIM == 3 ? (k >> 1) : 0));
  F.phi[c] += C.phi[q] - C.phi0[q];
  F.mu[c] += C.mu[q] - C.mu0[q];
  F.p[c] += C.p[q] - C.p0[q];
}

// phi^m and phi* on the coarse grid: mean of the children (once per step).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_restrict_coef(Level<T> F, Level<T> C) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= C.ncell) return;
  int I, J, KK;
  cell_ijk(q, C.nx, C.ny, I, J, KK);
  T a = 0, b = 0;
  const int kz = DIM == 3 ? 2 : 1;
  for (int dk = 0; dk < kz; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int c = (2 * I + di) + F.nx * ((2 * J + dj) + F.ny * (2 * KK + dk));
        a += F.phim[c];
        b += F.phis[c];
      }
  const T w = DIM == 3 ? T(0.125) : T(0.25);
  C.phim[q] = w * a;
  C.phis[q] = w * b;
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

// Partial sums of r_phi^2 + r_mu^2 + (s r_p)^2 over the fine grid, one per block.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_resid_partial(Level<T> L, Coefs<T> K, double* partials) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (c < L.ncell) {
    int i, j, k;
    cell_ijk(c, L.nx, L.ny, i, j, k);
    T n1, n2, n3;
    apply_N<T, DIM>(L, K, c, i, j, k, n1, n2, n3);
    double r1 = double(L.fphi[c] - n1), r2 = double(L.fmu[c] - n2);
    double r3 = double(K.s) * double(L.fp[c] - n3);
    acc[0] = r1 * r1 + r2 * r2 + r3 * r3;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// Sum the partials in a fixed order (deterministic), one block.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int nparts, double (&tot)[NV]) {
  for (int q = 0; q < NV; ++q) tot[q] = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int q = 0; q < NV; ++q) tot[q] += partials[b * NV + q];
  block_sum<NV>(tot);
}

// Finish the stopping norm.  mode 0: start of a step (records r0); mode 1:
// after a V-cycle (counts it).  Sets the while-loop condition of the step graph.
static __global__ void k_resid_finish(const double* partials, int nparts, int ncell, DevState* st,
                               cudaGraphConditionalHandle cond, int mode, int use_cond) {
  double tot[1];
  sum_partials<1>(partials, nparts, tot);
  if (threadIdx.x != 0) return;
  double r = sqrt(tot[0] / ncell);
  st->resid = r;
  unsigned int go = 0;
  if (st->failed == 0) {
    if (mode == 0) {
      st->r0 = r;
      st->vcycles = 0;
      go = (r > st->tol) ? 1u : 0u;
    } else {
      st->vcycles += 1;
      bool finite = isfinite(r);
      if (!finite || r > 1e8 * (st->r0 + 1.0)) {
        st->failed = 5;  // CHHS_ERR_DIVERGED
      } else if (r > st->tol) {
        if (st->vcycles >= st->max_v) st->failed = 4;  // CHHS_ERR_NOT_CONVERGED
        else go = 1u;
      }
    }
  }
  st->go = (int)go;
  if (use_cond) cudaGraphSetConditional(cond, go);
}

// ---------------------------------------------------------------- step frame

// phi* = 3/2 phi^m - 1/2 phi^{m-1} (Eq. 2.4); f_phi = phi^m;
// f_mu = -phi* - (1/4) eps^2 Lap_h phi^{m-1}; f_p = 0; initial guess
// phi = 2 phi^m - phi^{m-1} (mu and p keep the previous step's values).
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_setup(Level<double> L, const double* phimm1, double eps2,
                                                  const DevState* st) {
  if (st->failed) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
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
  L.fmu[c] = -ps - 0.25 * eps2 * L.ih2 * lap;
  L.fp[c] = 0.0;
  L.phi[c] = 2.0 * pm - pmm;
}

// Partial sums of v (NV = 1), one per block.
static __global__ void __launch_bounds__(kBlock) k_sum_partial(const double* v, int n, double* partials) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {c < n ? v[c] : 0.0};
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

static __global__ void k_mean_finish(const double* partials, int nparts, int n, DevState* st) {
  double tot[1];
  sum_partials<1>(partials, nparts, tot);
  if (threadIdx.x == 0) st->pmean = tot[0] / n;
}

// Accept the step: phi^{m-1} <- phi^m, phi^m <- phi^{m+1}, p <- p - mean(p).
static __global__ void __launch_bounds__(kBlock) k_advance(Level<double> L, double* phimm1, DevState* st) {
  if (st->failed) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) {
    st->steps_done += 1;
    st->vtotal += st->vcycles;
  }
  if (c >= L.ncell) return;
  phimm1[c] = L.phim[c];
  L.phim[c] = L.phi[c];
  L.p[c] -= st->pmean;
}

// ---------------------------------------------------------------- coarsest

// The coarsest grid (2^d cells for power-of-two grids) solved in one block:
// red-black sweeps until the residual has fallen by 1e-13 or stops falling.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_coarsest(Level<T> L, Coefs<T> K) {
  __shared__ double sh_r;
  double r0 = -1.0, prev = 0.0;
  for (int it = 0; it <= 2000; ++it) {
    double acc[1] = {0.0};
    for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
      int i, j, k;
      cell_ijk(c, L.nx, L.ny, i, j, k);
      T n1, n2, n3;
      apply_N<T, DIM>(L, K, c, i, j, k, n1, n2, n3);
      double r1 = double(L.fphi[c] - n1), r2 = double(L.fmu[c] - n2);
      double r3 = double(K.s) * double(L.fp[c] - n3);
      acc[0] += r1 * r1 + r2 * r2 + r3 * r3;
    }
    block_sum<1>(acc);
    if (threadIdx.x == 0) sh_r = sqrt(acc[0] / L.ncell);
    __syncthreads();
    double r = sh_r;
    __syncthreads();
    if (r0 < 0.0) r0 = r;
    if (!(r > 1e-13 * r0) || r < 1e-300) break;
    if (it > 50 && r > 0.999 * prev) break;
    prev = r;
    for (int colour = 0; colour < 2; ++colour) {
      for (int c = threadIdx.x; c < L.ncell; c += blockDim.x) {
        int i, j, k;
        cell_ijk(c, L.nx, L.ny, i, j, k);
        if (((i + j + k) & 1) != colour) continue;
        T phic = L.phi[c], muc = L.mu[c], pc = L.p[c], phimc = L.phim[c];
        Sums<T> S;
        face_sums<T, DIM>(L, K, c, i, j, k, phic, muc, pc, L.phis[c], S);
        T n1 = phic - K.s * L.ih2 * (S.Mdmu + S.adp);
        T n2 = muc - chi(phic, phimc) + K.e34 * L.ih2 * S.dphi;
        T n3 = -L.ih2 * (S.dp + K.gamma * S.admu);
        T R1 = L.fphi[c] - n1, R2 = L.fmu[c] - n2, R3 = L.fp[c] - n3;
        T inv_m = T(1) / T(S.m);
        T Ae = K.s * L.ih2 * (S.M - K.gamma * S.a * S.a * inv_m);
        T CD = K.s * S.a * inv_m;
        T G = K.gamma * L.ih2 * S.a;
        T B = dchi_da(phic, phimc) + K.e34 * L.ih2 * T(S.m);
        T dphi = (R1 - Ae * R2 - CD * R3) / (T(1) + Ae * B);
        T dmu = R2 + B * dphi;
        T dp = (R3 - G * dmu) * inv_m / L.ih2;
        L.phi[c] = phic + dphi;
        L.mu[c] = muc + dmu;
        L.p[c] = pc + dp;
      }
      __syncthreads();
    }
  }
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

static __global__ void k_energy_finish(const double* partials, int nparts, DevState* st) {
  double tot[6];
  sum_partials<6>(partials, nparts, tot);
  if (threadIdx.x == 0)
    for (int q = 0; q < 6; ++q) st->diag[q] = tot[q];
}

}  // namespace chhs_dev
