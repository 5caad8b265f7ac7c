// chhs_corr3.cuh -- the single-precision correction-form kernels of the 3D
// V-cycles (mixed-precision form), with the step's face coefficients
// recomputed from phi* in every pass instead of loaded.
//
// A colour pass of the stored-coefficient smoother (k_smooth) reads about 22
// arrays per cell (the state, the right-hand sides, phi^m, phi_b and 14 face
// and per-cell coefficient arrays); at 128^3 a level is 8.4 MB per array, so
// the finest passes stream ~200 MB each from HBM.  Recomputing the face
// values a_f = (phi*_c + phi*_e)/2 and M_f = 1 + gamma a_f^2, their sums and
// the smoother's constants (the formulas of coef_at) costs a few dozen
// single-precision operations and leaves 10 arrays to stream: phi, mu, p,
// the three right-hand sides, phi^m, phi*, phi_b (and the written state).
//
// Two transfers are folded into the passes around them:
//   - prolongation: the first post-smoothing pass (colour 0) reads every
//     value as e + P(e_c - e_c^0) (piecewise constant) and writes its cells
//     prolonged and smoothed; the second pass (colour 1) adds the correction
//     to its own cell only, whose neighbours are then final;
//   - the double-precision update of the mixed form: the last pass of the
//     finest level adds the finished correction to the double-precision
//     iterate, u <- u + e, for its own cell and for the cell of the other
//     colour beside it in x (whose correction the pass before finished).
#pragma once
#include "chhs_kernels.cuh"

namespace chhs_dev {

// Face data of cell c recomputed from phi*: neighbour index per face (c
// itself where the face is missing, so that every load is in bounds), a_f
// and M_f (zero on missing faces), their sums and the interior-face count.
template <int DIM>
struct FacesC {
  int e[2 * DIM];
  float a[2 * DIM], M[2 * DIM];
  float sM, sa;
  int m;
  unsigned in;  // bit q: face q is interior
};

template <int DIM>
__device__ __forceinline__ void faces_c(const Level<float>& L, const Coefs<float>& K, int c, int i, int j, int k,
                                        FacesC<DIM>& F) {
  const int sy = L.nx, sz = L.nx * L.ny;
  const bool in[6] = {i > 0, i + 1 < L.nx, j > 0, j + 1 < L.ny, k > 0, k + 1 < L.nz};
  const int off[6] = {-1, 1, -sy, sy, -sz, sz};
  const float pc = L.phis[c];
  F.sM = -0.f;
  F.sa = -0.f;
  F.m = 0;
  F.in = 0u;
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) {
    const int e = in[q] ? c + off[q] : c;
    const float af = 0.5f * (pc + L.phis[e]);
    F.e[q] = e;
    F.a[q] = in[q] ? af : 0.f;
    F.M[q] = in[q] ? 1.f + K.gamma * af * af : 0.f;
    F.sM += F.M[q];
    F.sa += F.a[q];
    F.m += in[q] ? 1 : 0;
    F.in |= in[q] ? (1u << q) : 0u;
  }
}

// Values of the correction at cell x = (i, j, k), with the prolongation
// P(e_c - e_c^0) of the next coarser level C added when `pro` is set.
struct Val3 {
  float phi, mu, p;
};

__device__ __forceinline__ Val3 read_val(const Level<float>& L, const Level<float>& C, int x, int i, int j, int k,
                                         bool pro) {
  Val3 v{L.phi[x], L.mu[x], L.p[x]};
  if (pro) {
    const int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
    v.phi += C.phi[q] - C.phi0[q];
    v.mu += C.mu[q] - C.mu0[q];
    v.p += C.p[q] - C.p0[q];
  }
  return v;
}

// Coordinates of the neighbour across face q (the cell itself on a missing face).
template <int DIM>
__device__ __forceinline__ void nb_coords(const FacesC<DIM>& F, int q, int i, int j, int k, int& a, int& b, int& d) {
  const bool in = (F.in >> q) & 1u;
  const int s = in ? ((q & 1) ? 1 : -1) : 0;
  a = i + ((q >> 1) == 0 ? s : 0);
  b = j + ((q >> 1) == 1 ? s : 0);
  d = k + ((q >> 1) == 2 ? s : 0);
}

// N(e) at cell c in correction form on explicitly given values: own value u,
// neighbour values nb[] (the cell itself on missing faces), base phi_b and
// phi^m at c.
template <int DIM>
__device__ __forceinline__ void n_corr(const Level<float>& L, const Coefs<float>& K, const FacesC<DIM>& F,
                                       const Val3& u, const Val3 (&nb)[2 * DIM], float phib, float pm, float& n1,
                                       float& n2, float& n3) {
  float Mp = -0.f, amu = -0.f, sphi = -0.f, sp = -0.f;
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) {
    const bool in = (F.in >> q) & 1u;
    Mp += F.M[q] * nb[q].mu;
    Mp += F.a[q] * nb[q].p;
    amu += F.a[q] * nb[q].mu;
    sphi += in ? nb[q].phi : -0.f;
    sp += in ? nb[q].p : -0.f;
  }
  const float mm = (float)F.m;
  const float chi_d = 0.25f * u.phi * (3.f * phib * phib + 2.f * phib * pm + pm * pm + (3.f * phib + pm) * u.phi +
                                       u.phi * u.phi);
  n1 = u.phi - L.sih2 * ((Mp - F.sM * u.mu) - F.sa * u.p);
  n2 = u.mu - chi_d + L.e34ih2 * (sphi - mm * u.phi);
  n3 = -L.ih2 * ((sp - mm * u.p) + K.gamma * (amu - F.sa * u.mu));
}

// One colour pass of the correction-form smoother on a single-precision
// level with recomputed coefficients (the update of cell_update: a Newton
// step on the cell's (phi, mu, p) with the pressure row eliminated).
//   rhs: complete the FAS right-hand side f += N(R u) at the pass's cells
//        first (the first pre-smoothing sweep on a coarse level);
//   pro: 1 = every value read with the prolongation added (first
//        post-smoothing pass), 2 = the own cell's only (second pass);
//   U:   when U.phi is set (the last pass on the finest level of the mixed
//        form), u <- u + e in double precision for the pass's cell and for
//        its x-neighbour of the other colour.
template <int DIM>
__device__ __forceinline__ void smooth_c_body(int bx, const Level<float>& L, const Level<float>& C,
                                              const Coefs<float>& K, int colour, int rhs, int pro,
                                              const Level<double>& U) {
  const int hw = (L.nx + 1) >> 1;
  const int t = bx * blockDim.x + threadIdx.x;
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
  const int i = 2 * ti + ((j + k + colour) & 1);
  const int i_other = 2 * ti + ((j + k + colour + 1) & 1);  // the other colour's cell of the x-pair
  if (i < L.nx) {
    const int c = i + L.nx * (j + L.ny * k);
    FacesC<DIM> F;
    faces_c<DIM>(L, K, c, i, j, k, F);
    const float pm = L.phim[c], phib = L.phib[c];
    float f1 = L.fphi[c], f2 = L.fmu[c], f3 = L.fp[c];
    if (rhs) {  // f += N(R u), R u = (phi0, mu0, p0) of this coarse level
      Val3 u0{L.phi0[c], L.mu0[c], L.p0[c]};
      Val3 nb0[2 * DIM];
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q) nb0[q] = Val3{L.phi0[F.e[q]], L.mu0[F.e[q]], L.p0[F.e[q]]};
      float n1, n2, n3;
      n_corr<DIM>(L, K, F, u0, nb0, phib, pm, n1, n2, n3);
      f1 += n1;
      f2 += n2;
      f3 += n3;
      L.fphi[c] = f1;
      L.fmu[c] = f2;
      L.fp[c] = f3;
    }
    const Val3 u = read_val(L, C, c, i, j, k, pro != 0);
    Val3 nb[2 * DIM];
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) {
      int a, b, d;
      nb_coords<DIM>(F, q, i, j, k, a, b, d);
      nb[q] = read_val(L, C, F.e[q], a, b, d, pro == 1);
    }
    float n1, n2, n3;
    n_corr<DIM>(L, K, F, u, nb, phib, pm, n1, n2, n3);
    const float R1 = f1 - n1, R2 = f2 - n2;
    const float im = rcp_approx((float)F.m);
    const float R3n = L.h2 * im * (f3 - n3);
    const float w = phib + u.phi;
    const float B = (0.75f * w + 0.5f * pm) * w + 0.25f * pm * pm + L.e34ih2 * (float)F.m;
    const float Ae = L.sih2 * (F.sM - K.gamma * F.sa * F.sa * im);
    const float Cc = L.sih2 * F.sa, Gn = K.gamma * F.sa * im;
    const float dphi = ((R1 - Ae * R2) - Cc * R3n) * rcp_approx(1.f + Ae * B);
    const float dmu = R2 + B * dphi;
    const float dp = R3n - Gn * dmu;
    const float ephi = u.phi + dphi, emu = u.mu + dmu, ep = u.p + dp;
    L.phi[c] = ephi;
    L.mu[c] = emu;
    L.p[c] = ep;
    if (U.phi) {
      U.phi[c] += (double)ephi;
      U.mu[c] += (double)emu;
      U.p[c] += (double)ep;
    }
  }
  if (U.phi && i_other < L.nx) {  // the other colour's cell: its correction is final
    const int c = i_other + L.nx * (j + L.ny * k);
    U.phi[c] += (double)L.phi[c];
    U.mu[c] += (double)L.mu[c];
    U.p[c] += (double)L.p[c];
  }
}

// At least 8 blocks of 128 threads per SM: 64 registers, no spills (left to
// itself the compiler takes 72-114 and the pass, which is bound by latency
// with the level's fields in L2, runs 4-35% slower on GB300).
template <int DIM>
__global__ void __launch_bounds__(kSmoothBlock, 8) k_smooth_c(const __grid_constant__ Level<float> L,
                                                           const __grid_constant__ Level<float> C, Coefs<float> K,
                                                           int colour, int rhs, int pro,
                                                           const __grid_constant__ Level<double> U) {
  pdl_enter();
  smooth_c_body<DIM>(blockIdx.x, L, C, K, colour, rhs, pro, U);
}

// Residual of the correction form and its restriction (k_residual_restrict's
// warp tiles of 16 x 2 / 8 x 2 x 2 fine cells, children summed by shuffles),
// with recomputed coefficients.  Writes u_c = u_c^0 = R e, f_c = R r and
// phi_b,c = R phi_b.
template <int DIM>
__device__ __forceinline__ void residual_restrict_c_body(int bx, const Level<float>& F, const Level<float>& C,
                                                         const Coefs<float>& K) {
  constexpr int TX = DIM == 3 ? 8 : 16;
  const int lane = threadIdx.x & 31;
  const int warp = (bx * blockDim.x + threadIdx.x) >> 5;
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
  float v[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) v[q] = 0.f;
  if (valid) {
    const int c = i + F.nx * (j + F.ny * k);
    FacesC<DIM> Fc;
    faces_c<DIM>(F, K, c, i, j, k, Fc);
    const Val3 u{F.phi[c], F.mu[c], F.p[c]};
    Val3 nb[2 * DIM];
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) nb[q] = Val3{F.phi[Fc.e[q]], F.mu[Fc.e[q]], F.p[Fc.e[q]]};
    const float phib = F.phib[c];
    float n1, n2, n3;
    n_corr<DIM>(F, K, Fc, u, nb, phib, F.phim[c], n1, n2, n3);
    v[0] = F.fphi[c] - n1;
    v[1] = F.fmu[c] - n2;
    v[2] = F.fp[c] - n3;
    v[3] = u.phi;
    v[4] = u.mu;
    v[5] = u.p;
    v[6] = phib;
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1);
    v[q] += __shfl_xor_sync(0xffffffffu, v[q], TX);
    if (DIM == 3) v[q] += __shfl_xor_sync(0xffffffffu, v[q], 16);
  }
  const bool leader = valid && (lane & 1) == 0 && ((lane / TX) & 1) == 0 && (DIM == 2 || lane < 16);
  if (!leader) return;
  const float w = DIM == 3 ? 0.125f : 0.25f;
  const int q = (i >> 1) + C.nx * ((j >> 1) + C.ny * (k >> 1));
  C.fphi[q] = w * v[0];
  C.fmu[q] = w * v[1];
  C.fp[q] = w * v[2];
  C.phi[q] = C.phi0[q] = w * v[3];
  C.mu[q] = C.mu0[q] = w * v[4];
  C.p[q] = C.p0[q] = w * v[5];
  C.phib[q] = w * v[6];
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_residual_restrict_c(const __grid_constant__ Level<float> F,
                                                                const __grid_constant__ Level<float> C,
                                                                Coefs<float> K) {
  pdl_enter();
  residual_restrict_c_body<DIM>(blockIdx.x, F, C, K);
}

}  // namespace chhs_dev
