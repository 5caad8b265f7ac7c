// chhs_tile.cuh -- several smoothing passes fused per shared-memory tile (2D).
//
// One block loads a tile of kTileW x kTileH cells of a level plus a halo of
// `halo` cells into shared memory and runs npass red-black colour passes of
// the smoother there.  Pass k (k = 1..npass) updates the cells of its colour
// in the tile grown by (halo - k) cells: every neighbour of those cells lies
// in the region that pass k-1 left exact, so after npass passes the tile
// grown by (halo - npass) cells holds exactly what npass grid-wide colour
// passes would give (cells of a colour are updated from the other colour's
// previous values either way).  The price is the recomputed halo cells; in
// single precision that is cheaper than the launches and global round trips
// it removes.
//
// Optional steps fused around the passes:
//   prolong  -- on load, u += P(u_c - u_c^0) (the FAS correction from the
//               next coarser level, piecewise constant);
//   rhs      -- before the first pass, f += N(u) on the cells that need it,
//               completing the FAS right-hand side R r + N_c(R u) (the tile's
//               u still equals R u at that point);
//   restrict -- after the passes (halo = npass + 1, so the ring around the
//               tile is exact too), the residual r = f - N(u) on the tile and
//               its restriction: u_c = u_c^0 = R u, f_c = R r, phi_b,c = R phi_b.
// The per-step face coefficients are recomputed from phi* in shared memory
// (cheap in single precision) instead of being read from global memory.
//
// A tile reads its halo from global memory while other tiles of the same
// launch write their results, so a launch never writes the arrays it reads:
// the pre-smoothing launch reads (phi, mu, p) and f and writes the second
// copy (phi2, mu2, p2) and the completed right-hand side (fc); the
// post-smoothing launch reads those and writes (phi, mu, p).  (Blocks of a
// launch are not all resident at once when other work shares the GPU.)
#pragma once
#include "chhs_kernels.cuh"

namespace chhs_dev {

constexpr int kTileW = 32, kTileH = 16;  // default tile interior (even, so restriction stays inside);
                                         // chhs_autotune may pick 32 x 32 or 64 x 16
constexpr int kTileThreads = 512;

template <bool CORR>
__host__ __device__ constexpr int tile_nfields() { return CORR ? 9 : 8; }

__host__ __device__ inline size_t tile_smem_bytes(int halo, int nfields, size_t elem, int tw = kTileW,
                                                  int th = kTileH) {
  return (size_t)(tw + 2 * halo) * (th + 2 * halo) * nfields * elem;
}

// Coefficients of cell (i, j) from phi* in shared memory: face values a_f,
// M_f for the interior faces, their sums and the smoother's Ae, C/Dn, G
// (the formulas of k_coef).
template <typename T>
struct LocalCoef {
  T aW, aE, aS, aN, MW, ME, MS, MN;  // zero on boundary faces
  T sM, sa, Ae, CD, G;
  int m;
};

template <typename T>
__device__ __forceinline__ void local_coef(const T* ps, int s, int SW, int i, int j, int nx, int ny,
                                           const Level<T>& L, const Coefs<T>& K, LocalCoef<T>& C) {
  const T pc = ps[s];
  // branch-free: a missing face reads the cell itself and gets a = M = 0
  auto face = [&](bool inside, int e, T& a, T& M) {
    const T af = T(0.5) * (pc + ps[inside ? e : s]);
    a = inside ? af : T(0);
    M = inside ? T(1) + K.gamma * af * af : T(0);
  };
  face(i > 0, s - 1, C.aW, C.MW);
  face(i + 1 < nx, s + 1, C.aE, C.ME);
  face(j > 0, s - SW, C.aS, C.MS);
  face(j + 1 < ny, s + SW, C.aN, C.MN);
  C.m = (i > 0) + (i + 1 < nx) + (j > 0) + (j + 1 < ny);
  C.sM = (C.MW + C.ME) + (C.MS + C.MN);
  C.sa = (C.aW + C.aE) + (C.aS + C.aN);
  const T im = inv_count<T>(C.m);
  C.Ae = L.sih2 * (C.sM - K.gamma * C.sa * C.sa * im);
  C.CD = K.s * C.sa * im;
  C.G = K.gamma * L.ih2 * C.sa;
}

// Where a tile launch writes its interior: (phi, mu, p) and, with rhs, the
// completed right-hand side.  On the finest level of the mixed form the
// post-smoothing launch instead adds the finished correction to the
// double-precision iterate (phi64, mu64, p64 non-null): u <- u + e.
template <typename T>
struct TileOut {
  T *phi, *mu, *p, *f1, *f2, *f3;
  double *phi64, *mu64, *p64;
};

// Shared-memory views of one tile's fields.
template <typename T, bool CORR>
struct TileView {
  T *phi, *mu, *p, *phim, *phis, *f1, *f2, *f3, *phib;
};

// N(u) at shared-memory cell s (global (i, j)).
template <typename T, bool CORR>
__device__ __forceinline__ void tile_N(const TileView<T, CORR>& V, int s, int SW, int i, int j, int nx, int ny,
                                       const Level<T>& L, const Coefs<T>& K, const LocalCoef<T>& C, T& n1, T& n2,
                                       T& n3) {
  T Mmu = 0, ap = 0, amu = 0, sphi = 0, sp = 0;
  // branch-free: a missing face (a = M = 0 from local_coef) reads the cell itself
  auto face = [&](bool inside, int e, T a, T M) {
    const int es = inside ? e : s;
    const T mue = V.mu[es], pe = V.p[es], phie = V.phi[es];
    Mmu += M * mue;
    ap += a * pe;
    amu += a * mue;
    sphi += inside ? phie : T(0);
    sp += inside ? pe : T(0);
  };
  face(i > 0, s - 1, C.aW, C.MW);
  face(i + 1 < nx, s + 1, C.aE, C.ME);
  face(j > 0, s - SW, C.aS, C.MS);
  face(j + 1 < ny, s + SW, C.aN, C.MN);
  const T phic = V.phi[s], muc = V.mu[s], pc = V.p[s], pm = V.phim[s], mm = count_value<T>(C.m);
  T chi_v;
  if (CORR) {
    T b = V.phib[s];
    chi_v = T(0.25) * phic * (T(3) * b * b + T(2) * b * pm + pm * pm + (T(3) * b + pm) * phic + phic * phic);
  } else {
    chi_v = chi(phic, pm);
  }
  n1 = phic - L.sih2 * ((Mmu - C.sM * muc) + (ap - C.sa * pc));
  n2 = muc - chi_v + L.e34ih2 * (sphi - mm * phic);
  n3 = -L.ih2 * ((sp - mm * pc) + K.gamma * (amu - C.sa * muc));
}

template <typename T, bool CORR>
__device__ __forceinline__ void tile_body(int bx, int by, const Level<T>& L, const Level<T>& Cl,
                                          const Coefs<T>& K, int npass, int halo, int rhs, int prolong,
                                          int restrict_out, const TileOut<T>& out, int tw = kTileW,
                                          int th = kTileH) {
  // The tiles serve the correction-form (single-precision) levels only: the
  // plain form's right-hand side f_mu carries the shift of cubic_P, which
  // tile_N does not.
  static_assert(CORR, "k_tile runs the correction form only");
  extern __shared__ __align__(16) unsigned char tile_smem[];
  const int SW = tw + 2 * halo, SH = th + 2 * halo, SN = SW * SH;
  TileView<T, CORR> V;
  {
    T* base = reinterpret_cast<T*>(tile_smem);
    V.phi = base; V.mu = base + SN; V.p = base + 2 * SN; V.phim = base + 3 * SN; V.phis = base + 4 * SN;
    V.f1 = base + 5 * SN; V.f2 = base + 6 * SN; V.f3 = base + 7 * SN;
    V.phib = CORR ? base + 8 * SN : nullptr;
  }
  const int nx = L.nx, ny = L.ny;
  const int tx0 = bx * tw, ty0 = by * th;  // tile origin (global)
  const int gx0 = tx0 - halo, gy0 = ty0 - halo;                      // shared-memory origin (global)

  // load the tile and its halo (cells outside the domain are never read);
  // thread-to-cell maps use small_div (every index here is below 2^21)
  const float rSW = __frcp_rn((float)SW);
  for (int s = threadIdx.x; s < SN; s += blockDim.x) {
    int sy = small_div(s, rSW), sx = s - sy * SW;
    int i = gx0 + sx, j = gy0 + sy;
    if (i < 0 || j < 0 || i >= nx || j >= ny) continue;
    int c = i + nx * j;
    T phi = L.phi[c], mu = L.mu[c], p = L.p[c];
    if (prolong) {
      int q = (i >> 1) + Cl.nx * (j >> 1);
      phi += Cl.phi[q] - Cl.phi0[q];
      mu += Cl.mu[q] - Cl.mu0[q];
      p += Cl.p[q] - Cl.p0[q];
    }
    V.phi[s] = phi;
    V.mu[s] = mu;
    V.p[s] = p;
    V.phim[s] = L.phim[c];
    V.phis[s] = L.phis[c];
    V.f1[s] = L.fphi[c];
    V.f2[s] = L.fmu[c];
    V.f3[s] = L.fp[c];
    if (CORR) V.phib[s] = L.phib[c];
  }
  __syncthreads();

  // the cells of region "tile grown by g" inside the domain: [x0, x1) x [y0, y1)
  auto region = [&](int g, int& x0, int& x1, int& y0, int& y1) {
    x0 = max(tx0 - g, 0);
    x1 = min(tx0 + tw + g, nx);
    y0 = max(ty0 - g, 0);
    y1 = min(ty0 + th + g, ny);
  };

  if (rhs) {  // f += N(R u) wherever pass 1 needs f
    int x0, x1, y0, y1;
    region(halo - 1, x0, x1, y0, y1);
    const int w = x1 - x0, total = w * (y1 - y0);
    const float rw = __frcp_rn((float)w);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int q = small_div(t, rw);
      int j = y0 + q, i = x0 + (t - q * w);
      int s = (i - gx0) + SW * (j - gy0);
      LocalCoef<T> C;
      local_coef(V.phis, s, SW, i, j, nx, ny, L, K, C);
      T n1, n2, n3;
      tile_N<T, CORR>(V, s, SW, i, j, nx, ny, L, K, C, n1, n2, n3);
      V.f1[s] += n1;
      V.f2[s] += n2;
      V.f3[s] += n3;
    }
    __syncthreads();
  }

  for (int k = 1; k <= npass; ++k) {
    const int colour = (k - 1) & 1;
    int x0, x1, y0, y1;
    region(halo - k, x0, x1, y0, y1);
    const int hw = (x1 - x0 + 1) >> 1, total = hw * (y1 - y0);
    const float rhw = __frcp_rn((float)hw);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int q = small_div(t, rhw);
      int j = y0 + q;
      int i = x0 + 2 * (t - q * hw);
      i += (i + j + colour) & 1;
      if (i >= x1) continue;
      int s = (i - gx0) + SW * (j - gy0);
      LocalCoef<T> C;
      local_coef(V.phis, s, SW, i, j, nx, ny, L, K, C);
      T n1, n2, n3;
      tile_N<T, CORR>(V, s, SW, i, j, nx, ny, L, K, C, n1, n2, n3);
      const T phic = V.phi[s], pm = V.phim[s];
      T R1 = V.f1[s] - n1, R2 = V.f2[s] - n2, R3 = V.f3[s] - n3;
      T dchi = CORR ? dchi_da(V.phib[s] + phic, pm) : dchi_da(phic, pm);
      T B = dchi + L.e34ih2 * count_value<T>(C.m);
      T dphi = (R1 - C.Ae * R2 - C.CD * R3) * rcp_approx(T(1) + C.Ae * B);
      T dmu = R2 + B * dphi;
      T dp = (R3 - C.G * dmu) * (L.h2 * inv_count<T>(C.m));
      V.phi[s] = phic + dphi;
      V.mu[s] += dmu;
      V.p[s] += dp;
    }
    __syncthreads();
  }

  // write the tile back
  {
    int x0, x1, y0, y1;
    region(0, x0, x1, y0, y1);
    const int w = x1 - x0, total = w * (y1 - y0);
    const float rw = __frcp_rn((float)w);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int q = small_div(t, rw);
      int j = y0 + q, i = x0 + (t - q * w);
      int s = (i - gx0) + SW * (j - gy0), c = i + nx * j;
      if (out.phi64) {
        out.phi64[c] += (double)V.phi[s];
        out.mu64[c] += (double)V.mu[s];
        out.p64[c] += (double)V.p[s];
      } else {
        out.phi[c] = V.phi[s];
        out.mu[c] = V.mu[s];
        out.p[c] = V.p[s];
      }
      if (rhs) {
        out.f1[c] = V.f1[s];
        out.f2[c] = V.f2[s];
        out.f3[c] = V.f3[s];
      }
    }
  }

  if (restrict_out) {
    // residual on the tile and its restriction: one thread per fine cell,
    // the four children of a coarse cell in adjacent lanes (child d = t mod 4),
    // summed by shuffles in a fixed order; the round count is uniform so
    // every thread takes part in the shuffles
    constexpr int NV = CORR ? 7 : 6;
    const int cw = tw / 2, chh = th / 2, total = 4 * cw * chh;
    for (int r = 0; r < total; r += blockDim.x) {
      const int t = r + threadIdx.x, qq = t >> 2, d = t & 3;
      const int I = (tx0 >> 1) + qq % cw, J = (ty0 >> 1) + qq / cw;
      const bool act = t < total && I < Cl.nx && J < Cl.ny;
      T v[NV];
#pragma unroll
      for (int m = 0; m < NV; ++m) v[m] = T(0);
      if (act) {
        const int i = 2 * I + (d & 1), j = 2 * J + (d >> 1);
        const int s = (i - gx0) + SW * (j - gy0);
        LocalCoef<T> C;
        local_coef(V.phis, s, SW, i, j, nx, ny, L, K, C);
        T n1, n2, n3;
        tile_N<T, CORR>(V, s, SW, i, j, nx, ny, L, K, C, n1, n2, n3);
        v[0] = V.f1[s] - n1;
        v[1] = V.f2[s] - n2;
        v[2] = V.f3[s] - n3;
        v[3] = V.phi[s];
        v[4] = V.mu[s];
        v[5] = V.p[s];
        if (CORR) v[NV - 1] = V.phib[s];
      }
#pragma unroll
      for (int o = 1; o < 4; o <<= 1)
#pragma unroll
        for (int m = 0; m < NV; ++m) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
      if (act && d == 0) {
        const int q = I + Cl.nx * J;
        Cl.fphi[q] = T(0.25) * v[0];
        Cl.fmu[q] = T(0.25) * v[1];
        Cl.fp[q] = T(0.25) * v[2];
        Cl.phi[q] = Cl.phi0[q] = T(0.25) * v[3];
        Cl.mu[q] = Cl.mu0[q] = T(0.25) * v[4];
        Cl.p[q] = Cl.p0[q] = T(0.25) * v[5];
        if (CORR) Cl.phib[q] = T(0.25) * v[NV - 1];
      }
    }
  }
}

// gate (nullable): the run's loop flag; the launch does nothing once the
// run has stopped iterating (a run of a batch that has converged).
template <typename T, bool CORR>
__global__ void __launch_bounds__(kTileThreads) k_tile(const __grid_constant__ Level<T> L,
                                                      const __grid_constant__ Level<T> Cl, Coefs<T> K, int npass,
                                                      int halo, int rhs, int prolong, int restrict_out,
                                                      const __grid_constant__ TileOut<T> out, const int* gate,
                                                      int tw, int th) {
  pdl_enter();
  if (gate && *(volatile const int*)gate == 0) return;
  tile_body<T, CORR>(blockIdx.x, blockIdx.y, L, Cl, K, npass, halo, rhs, prolong, restrict_out, out, tw, th);
}

}  // namespace chhs_dev
