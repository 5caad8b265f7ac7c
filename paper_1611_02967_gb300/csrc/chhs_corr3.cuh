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

// The cell's Newton step in correction form from its residual rows R1, R2,
// R3 (the pressure row eliminated, as in cell_update): the updated values.
template <int DIM>
__device__ __forceinline__ Val3 corr_newton(const Level<float>& L, const Coefs<float>& K, const FacesC<DIM>& F,
                                            const Val3& u, float phib, float pm, float R1, float R2, float R3) {
  const float im = rcp_approx((float)F.m);
  const float R3n = L.h2 * im * R3;
  const float w = phib + u.phi;
  const float B = (0.75f * w + 0.5f * pm) * w + 0.25f * pm * pm + L.e34ih2 * (float)F.m;
  const float Ae = L.sih2 * (F.sM - K.gamma * F.sa * F.sa * im);
  const float Cc = L.sih2 * F.sa, Gn = K.gamma * F.sa * im;
  const float dphi = ((R1 - Ae * R2) - Cc * R3n) * rcp_approx(1.f + Ae * B);
  const float dmu = R2 + B * dphi;
  const float dp = R3n - Gn * dmu;
  return Val3{u.phi + dphi, u.mu + dmu, u.p + dp};
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
    const Val3 e = corr_newton<DIM>(L, K, F, u, phib, pm, f1 - n1, f2 - n2, f3 - n3);
    const float ephi = e.phi, emu = e.mu, ep = e.p;
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

// Face data of a cell from its phi* value pc and its neighbours' pe[] (the
// cell's own value where in[q] is false), as faces_c forms it from indices
// (the x-quad passes and the restriction).
template <int DIM>
__device__ __forceinline__ void faces_vals(const Coefs<float>& K, float pc, const float (&pe)[6], const bool (&in)[6],
                                           FacesC<DIM>& F) {
  F.sM = -0.f;
  F.sa = -0.f;
  F.m = 0;
  F.in = 0u;
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) {
    const float af = 0.5f * (pc + pe[q]);
    F.e[q] = 0;
    F.a[q] = in[q] ? af : 0.f;
    F.M[q] = in[q] ? 1.f + K.gamma * af * af : 0.f;
    F.sM += F.M[q];
    F.sa += F.a[q];
    F.m += in[q] ? 1 : 0;
    F.in |= in[q] ? (1u << q) : 0u;
  }
}

// ------------------------------------------------------------ x-quad passes
//
// The 3D colour pass above with each lane on four consecutive cells of a row,
// 4q .. 4q+3, on levels whose nx is a multiple of 4.  The lane updates the two
// cells of the pass's colour among them, 4q+s and 4q+s+2 (s = (j + k +
// colour) & 1), and reads every field as 16-byte vectors: the quad, the quads
// beside it in y and z, and the one x neighbour outside the quad (4q-1 when
// s = 0, 4q+4 when s = 1) as a single value -- 6 load instructions per field
// for two updated cells where one cell per lane takes 7 for one, and the
// index arithmetic shared by both.  Each cell's arithmetic is that of
// smooth_c_body in the same order, missing faces included (the cell's own
// value under a zero coefficient), so the results are the same bit for bit.
// The state is written back as whole quads, the other colour's cells with
// the values the pass read (unchanged in memory during the pass).

// A field's values around an x-quad: the quad (o), the quads beside it in y
// and z (the quad itself on a missing face) and the outside x neighbour (e;
// the cell itself at the domain's end).
struct Quad {
  float4 o, ym, yp, zm, zp;
  float e;
};

struct QuadAt {
  int c4;       // first cell of the quad (a multiple of 4)
  int sy, sz;   // strides of y and z
  int xe;       // index of the outside x neighbour
  int s;        // the pass's cells are 4q+s and 4q+s+2
  bool ym, yp, zm, zp, xin;  // faces present; xin: the outside x neighbour exists
};

__device__ __forceinline__ float4 ld4(const float* a, int x) { return *reinterpret_cast<const float4*>(a + x); }

__device__ __forceinline__ Quad load_quad(const float* a, const QuadAt& Q) {
  Quad r;
  r.o = ld4(a, Q.c4);
  r.ym = Q.ym ? ld4(a, Q.c4 - Q.sy) : r.o;
  r.yp = Q.yp ? ld4(a, Q.c4 + Q.sy) : r.o;
  r.zm = Q.zm ? ld4(a, Q.c4 - Q.sz) : r.o;
  r.zp = Q.zp ? ld4(a, Q.c4 + Q.sz) : r.o;
  r.e = Q.xin ? a[Q.xe] : (Q.s ? r.o.w : r.o.x);
  return r;
}

// Coarse cells of the prolongation P(e_c - e_c^0) for a quad: the coarse
// x-pair 2q, 2q+1 of the quad's row and of the rows beside it in y and z
// (the quad's own where a face is missing), and of the outside x neighbour.
struct QuadCoarse {
  int o, ym, yp, zm, zp, e;
};

__device__ __forceinline__ float2 coarse_diff2(const float* cn, const float* c0, int x) {
  const float2 a = *reinterpret_cast<const float2*>(cn + x), b = *reinterpret_cast<const float2*>(c0 + x);
  return make_float2(a.x - b.x, a.y - b.y);
}

__device__ __forceinline__ void add_diff(float4& v, float2 d) {
  v.x += d.x;
  v.y += d.x;
  v.z += d.y;
  v.w += d.y;
}

// Every value of X read with the prolongation added (the first
// post-smoothing pass); dO returns the quad's own coarse differences.
__device__ __forceinline__ void prolong_quad(Quad& X, const float* cn, const float* c0, const QuadCoarse& P,
                                             const QuadAt& Q, float2& dO) {
  dO = coarse_diff2(cn, c0, P.o);
  add_diff(X.o, dO);
  add_diff(X.ym, coarse_diff2(cn, c0, P.ym));
  add_diff(X.yp, coarse_diff2(cn, c0, P.yp));
  add_diff(X.zm, coarse_diff2(cn, c0, P.zm));
  add_diff(X.zp, coarse_diff2(cn, c0, P.zp));
  X.e += Q.xin ? cn[P.e] - c0[P.e] : (Q.s ? dO.y : dO.x);
}

// RHS: complete the FAS right-hand side first (as rhs in smooth_c_body);
// PRO: 1 = every value read with the prolongation added, 2 = the pass's own
// cells only (as pro); U: as in smooth_c_body, here for all four cells of
// the quad (the other colour's two are final since the previous pass).
template <int RHS, int PRO>
__device__ __forceinline__ void smooth_c4_body(const Level<float>& L, const Level<float>& C, const Coefs<float>& K,
                                               int colour, const Level<double>& U, int tile) {
  // the block's brick of quads: 2^lq quads in x, 2^ly rows, 2^lz planes
  const int nq = L.nx >> 2;
  const int lq = tile & 15, ly = (tile >> 4) & 15, lz = tile >> 8;
  const int q = ((int)blockIdx.x << lq) + (threadIdx.x & ((1 << lq) - 1));
  const int j = ((int)blockIdx.y << ly) + ((threadIdx.x >> lq) & ((1 << ly) - 1));
  const int k = ((int)blockIdx.z << lz) + (threadIdx.x >> (lq + ly));
  if (q >= nq || j >= L.ny || k >= L.nz) return;
  const int row = j + L.ny * k;
  QuadAt Q;
  Q.s = (j + k + colour) & 1;
  Q.sy = L.nx;
  Q.sz = L.nx * L.ny;
  Q.c4 = 4 * q + L.nx * row;
  Q.ym = j > 0;
  Q.yp = j + 1 < L.ny;
  Q.zm = k > 0;
  Q.zp = k + 1 < L.nz;
  Q.xin = Q.s ? 4 * q + 4 < L.nx : q > 0;
  Q.xe = Q.s ? Q.c4 + 4 : Q.c4 - 1;

  const Quad S = load_quad(L.phis, Q);
  Quad P = load_quad(L.phi, Q), M = load_quad(L.mu, Q), R = load_quad(L.p, Q);
  const float4 pm4 = ld4(L.phim, Q.c4), pb4 = ld4(L.phib, Q.c4);
  float4 f1 = ld4(L.fphi, Q.c4), f2 = ld4(L.fmu, Q.c4), f3 = ld4(L.fp, Q.c4);
  Quad P0, M0, R0;
  if (RHS) {
    P0 = load_quad(L.phi0, Q);
    M0 = load_quad(L.mu0, Q);
    R0 = load_quad(L.p0, Q);
  }
  float4 outP = P.o, outM = M.o, outR = R.o;  // written back: the other colour's cells as read
  float2 dP = make_float2(0.f, 0.f), dM = dP, dR = dP;
  if (PRO) {
    QuadCoarse Pc;
    auto crow = [&](int jj, int kk) { return C.nx * ((jj >> 1) + C.ny * (kk >> 1)) + 2 * q; };
    Pc.o = crow(j, k);
    Pc.ym = crow(Q.ym ? j - 1 : j, k);
    Pc.yp = crow(Q.yp ? j + 1 : j, k);
    Pc.zm = crow(j, Q.zm ? k - 1 : k);
    Pc.zp = crow(j, Q.zp ? k + 1 : k);
    Pc.e = Pc.o + (Q.s ? 2 : -1);
    if (PRO == 1) {
      prolong_quad(P, C.phi, C.phi0, Pc, Q, dP);
      prolong_quad(M, C.mu, C.mu0, Pc, Q, dM);
      prolong_quad(R, C.p, C.p0, Pc, Q, dR);
    } else {
      dP = coarse_diff2(C.phi, C.phi0, Pc.o);
      dM = coarse_diff2(C.mu, C.mu0, Pc.o);
      dR = coarse_diff2(C.p, C.p0, Pc.o);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // the cells 4q+s, then 4q+s+2
    auto at = [&](const float4& v) { return h ? (Q.s ? v.w : v.z) : (Q.s ? v.y : v.x); };
    auto xm = [&](const Quad& X) { return h ? (Q.s ? X.o.z : X.o.y) : (Q.s ? X.o.x : X.e); };
    auto xp = [&](const Quad& X) { return h ? (Q.s ? X.e : X.o.w) : (Q.s ? X.o.z : X.o.y); };
    auto put = [&](float4& v, float x) {
      if (h) {
        v.w = Q.s ? x : v.w;
        v.z = Q.s ? v.z : x;
      } else {
        v.y = Q.s ? x : v.y;
        v.x = Q.s ? v.x : x;
      }
    };
    auto nbs = [&](const Quad& A, const Quad& B, const Quad& D, Val3 (&nb)[6]) {
      nb[0] = Val3{xm(A), xm(B), xm(D)};
      nb[1] = Val3{xp(A), xp(B), xp(D)};
      nb[2] = Val3{at(A.ym), at(B.ym), at(D.ym)};
      nb[3] = Val3{at(A.yp), at(B.yp), at(D.yp)};
      nb[4] = Val3{at(A.zm), at(B.zm), at(D.zm)};
      nb[5] = Val3{at(A.zp), at(B.zp), at(D.zp)};
    };
    const bool in[6] = {h || Q.s || Q.xin, !h || !Q.s || Q.xin, Q.ym, Q.yp, Q.zm, Q.zp};
    const float pe[6] = {xm(S), xp(S), at(S.ym), at(S.yp), at(S.zm), at(S.zp)};
    FacesC<3> F;
    faces_vals<3>(K, at(S.o), pe, in, F);
    const float pm = at(pm4), phib = at(pb4);
    float g1 = at(f1), g2 = at(f2), g3 = at(f3);
    float n1, n2, n3;
    if (RHS) {  // f += N(R u), R u = (phi0, mu0, p0) of this coarse level
      const Val3 u0{at(P0.o), at(M0.o), at(R0.o)};
      Val3 nb0[6];
      nbs(P0, M0, R0, nb0);
      n_corr<3>(L, K, F, u0, nb0, phib, pm, n1, n2, n3);
      g1 += n1;
      g2 += n2;
      g3 += n3;
      put(f1, g1);
      put(f2, g2);
      put(f3, g3);
    }
    Val3 u{at(P.o), at(M.o), at(R.o)};
    if (PRO == 2) {
      u.phi += h ? dP.y : dP.x;
      u.mu += h ? dM.y : dM.x;
      u.p += h ? dR.y : dR.x;
    }
    Val3 nb[6];
    nbs(P, M, R, nb);
    n_corr<3>(L, K, F, u, nb, phib, pm, n1, n2, n3);
    const Val3 e = corr_newton<3>(L, K, F, u, phib, pm, g1 - n1, g2 - n2, g3 - n3);
    put(outP, e.phi);
    put(outM, e.mu);
    put(outR, e.p);
  }
  if (RHS) {
    *reinterpret_cast<float4*>(L.fphi + Q.c4) = f1;
    *reinterpret_cast<float4*>(L.fmu + Q.c4) = f2;
    *reinterpret_cast<float4*>(L.fp + Q.c4) = f3;
  }
  *reinterpret_cast<float4*>(L.phi + Q.c4) = outP;
  *reinterpret_cast<float4*>(L.mu + Q.c4) = outM;
  *reinterpret_cast<float4*>(L.p + Q.c4) = outR;
  if (U.phi) {  // u <- u + e over the whole quad
    auto upd = [&](double* a, const float4& v) {
      double2* d = reinterpret_cast<double2*>(a + Q.c4);
      double2 lo = d[0], hi = d[1];
      lo.x += (double)v.x;
      lo.y += (double)v.y;
      hi.x += (double)v.z;
      hi.y += (double)v.w;
      d[0] = lo;
      d[1] = hi;
    };
    upd(U.phi, outP);
    upd(U.mu, outM);
    upd(U.p, outR);
  }
}

// Bricks of quads per block (kSmoothBlock = 2^7 threads): 2^lq quads in x with
// 2^lq the smallest power of two >= nx/4 up to 32, and the remaining factor
// split between y and z (z the smaller), packed as lq | ly << 4 | lz << 8,
// so that the warps of a block read each other's y and z neighbour rows
// (L1 hits) instead of rows of other blocks.
__host__ __device__ inline int quad_tile(int nx) {
  const int nq = nx / 4;
  int lq = 0;
  while ((1 << lq) < nq && lq < 5) ++lq;
  const int rem = 7 - lq, lz = rem >> 1;
  return lq | (rem - lz) << 4 | lz << 8;
}
__host__ __device__ inline dim3 quad_grid(int nx, int ny, int nz) {
  const int t = quad_tile(nx), lq = t & 15, ly = (t >> 4) & 15, lz = t >> 8;
  return dim3((unsigned)((nx / 4 + (1 << lq) - 1) >> lq), (unsigned)((ny + (1 << ly) - 1) >> ly),
              (unsigned)((nz + (1 << lz) - 1) >> lz));
}

// Launched on quad_grid with kSmoothBlock threads.  The plain pass fits 80 registers
// without spills (6 blocks of 128 threads per SM); the passes that also read
// the coarse level or R u, 128 (4 blocks).
template <int RHS, int PRO>
__global__ void __launch_bounds__(kSmoothBlock, (RHS || PRO) ? 4 : 6) k_smooth_c4(const __grid_constant__ Level<float> L,
                                                            const __grid_constant__ Level<float> C, Coefs<float> K,
                                                            int colour, const __grid_constant__ Level<double> U,
                                                            int tile) {
  pdl_enter();
  smooth_c4_body<RHS, PRO>(L, C, K, colour, U, tile);
}

// ---------------------------------------------------------------- restriction

// Warps of k_residual_restrict_c on an nx x ny (x nz) level: each covers 2 *
// rr_c_pairs(dim) x 2 (x 2) fine cells, a lane an x-pair of them.
__host__ __device__ constexpr int rr_c_pairs(int dim) { return dim == 3 ? 8 : 16; }
__host__ __device__ inline long long rr_c_warps(int dim, int nx, int ny, int nz) {
  const int px = rr_c_pairs(dim);
  return (long long)((nx + 2 * px - 1) / (2 * px)) * (ny / 2) * (dim == 3 ? nz / 2 : 1);
}

// Residual of the correction form and its restriction, with recomputed
// coefficients.  A lane takes the x-pair (i, i+1), i even -- two children of
// one coarse cell -- and reads every field as float2 pairs (the pair, and
// the pairs beside it in y and z; the two x neighbours outside the pair as
// single values), so a warp's loads are 8-byte vector loads over 2 * 8 x 2 x
// 2 (3D) or 2 * 16 x 2 (2D) fine cells.  The pair's two residuals are added
// in the lane, then the other children by shuffles in y and z (the order of
// the additions of one lane per cell and shuffles over x, y, z).  Writes
// u_c = u_c^0 = R e, f_c = R r and phi_b,c = R phi_b.
template <int DIM>
__device__ __forceinline__ void residual_restrict_c_body(int bx, const Level<float>& F, const Level<float>& C,
                                                         const Coefs<float>& K) {
  constexpr int PX = rr_c_pairs(DIM);
  const int lane = threadIdx.x & 31;
  const int warp = (bx * blockDim.x + threadIdx.x) >> 5;
  const int tiles_x = (F.nx + 2 * PX - 1) / (2 * PX);
  const int tiles_y = F.ny >> 1;
  const int tiles_z = DIM == 3 ? (F.nz >> 1) : 1;
  if (warp >= tiles_x * tiles_y * tiles_z) return;  // whole warp
  const int tx = warp % tiles_x;
  const int rest = warp / tiles_x;
  const int ty = rest % tiles_y, tz = rest / tiles_y;
  const int i = tx * 2 * PX + 2 * (lane % PX);  // the pair (i, i + 1); nx is even
  const int j = 2 * ty + ((lane / PX) & 1);
  const int k = DIM == 3 ? 2 * tz + (lane >> 4) : 0;
  const bool valid = i < F.nx;
  float v[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) v[q] = 0.f;
  if (valid) {
    const int c = i + F.nx * (j + F.ny * k);  // even
    const int sy = F.nx, sz = F.nx * F.ny;
    const bool xm = i > 0, xp = i + 2 < F.nx, ym = j > 0, yp = j + 1 < F.ny;
    const bool zm = DIM == 3 && k > 0, zp = DIM == 3 && k + 1 < F.nz;
    auto ld2 = [](const float* a, int x) { return *reinterpret_cast<const float2*>(a + x); };
    // the pair and its y/z neighbour pairs (the pair itself on a missing face)
    auto pairs = [&](const float* a, float2 (&P)[5]) {
      P[0] = ld2(a, c);
      P[1] = ym ? ld2(a, c - sy) : P[0];
      P[2] = yp ? ld2(a, c + sy) : P[0];
      P[3] = zm ? ld2(a, c - sz) : P[0];
      P[4] = zp ? ld2(a, c + sz) : P[0];
    };
    float2 S[5], Ph[5], Mu[5], Pr[5];
    pairs(F.phis, S);
    pairs(F.phi, Ph);
    pairs(F.mu, Mu);
    pairs(F.p, Pr);
    const float sxm = xm ? F.phis[c - 1] : S[0].x, sxp = xp ? F.phis[c + 2] : S[0].y;
    const Val3 uxm = xm ? Val3{F.phi[c - 1], F.mu[c - 1], F.p[c - 1]} : Val3{Ph[0].x, Mu[0].x, Pr[0].x};
    const Val3 uxp = xp ? Val3{F.phi[c + 2], F.mu[c + 2], F.p[c + 2]} : Val3{Ph[0].y, Mu[0].y, Pr[0].y};
    const float2 f1 = ld2(F.fphi, c), f2 = ld2(F.fmu, c), f3 = ld2(F.fp, c), pm = ld2(F.phim, c),
                 pb = ld2(F.phib, c);
    const bool yzin[4] = {ym, yp, zm, zp};
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // the pair's cells, i then i + 1
      auto cx = [h](const float2& a) { return h ? a.y : a.x; };
      const bool in[6] = {h ? true : xm, h ? xp : true, yzin[0], yzin[1], yzin[2], yzin[3]};
      const Val3 u{cx(Ph[0]), cx(Mu[0]), cx(Pr[0])};
      const Val3 other{h ? Ph[0].x : Ph[0].y, h ? Mu[0].x : Mu[0].y, h ? Pr[0].x : Pr[0].y};
      const float pc = cx(S[0]);
      float pe[6];
      Val3 nb[2 * DIM];
      pe[0] = h ? S[0].x : sxm;
      pe[1] = h ? sxp : S[0].y;
      nb[0] = h ? other : uxm;
      nb[1] = h ? uxp : other;
#pragma unroll
      for (int q = 2; q < 2 * DIM; ++q) {
        pe[q] = cx(S[q - 1]);
        nb[q] = Val3{cx(Ph[q - 1]), cx(Mu[q - 1]), cx(Pr[q - 1])};
      }
      if (DIM == 2) pe[4] = pe[5] = pc;
      FacesC<DIM> Fc;
      faces_vals<DIM>(K, pc, pe, in, Fc);
      const float phib = cx(pb);
      float n1, n2, n3;
      n_corr<DIM>(F, K, Fc, u, nb, phib, cx(pm), n1, n2, n3);
      const float r[7] = {cx(f1) - n1, cx(f2) - n2, cx(f3) - n3, u.phi, u.mu, u.p, phib};
#pragma unroll
      for (int q = 0; q < 7; ++q) v[q] = h ? v[q] + r[q] : r[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    v[q] += __shfl_xor_sync(0xffffffffu, v[q], PX);
    if (DIM == 3) v[q] += __shfl_xor_sync(0xffffffffu, v[q], 16);
  }
  const bool leader = valid && ((lane / PX) & 1) == 0 && (DIM == 2 || lane < 16);
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
