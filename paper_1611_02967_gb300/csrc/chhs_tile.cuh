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
#pragma once
#include "chhs_kernels.cuh"

namespace chhs_dev {

constexpr int kTileW = 32, kTileH = 16;  // tile interior (even, so restriction stays inside)
constexpr int kTileThreads = 256;

template <bool CORR>
__host__ __device__ constexpr int tile_nfields() { return CORR ? 9 : 8; }

__host__ __device__ inline size_t tile_smem_bytes(int halo, int nfields, size_t elem) {
  return (size_t)(kTileW + 2 * halo) * (kTileH + 2 * halo) * nfields * elem;
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
  auto face = [&](bool inside, int e, T& a, T& M) {
    if (inside) {
      a = T(0.5) * (pc + ps[e]);
      M = T(1) + K.gamma * a * a;
    } else {
      a = T(0);
      M = T(0);
    }
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
  auto face = [&](bool inside, int e, T a, T M) {
    if (!inside) return;
    T mue = V.mu[e], pe = V.p[e];
    Mmu += M * mue;
    ap += a * pe;
    amu += a * mue;
    sphi += V.phi[e];
    sp += pe;
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
__global__ void __launch_bounds__(kTileThreads) k_tile(Level<T> L, Level<T> Cl, Coefs<T> K, int npass,
                                                      int halo, int rhs, int prolong, int restrict_out) {
  // The tiles serve the correction-form (single-precision) levels only: the
  // plain form's right-hand side f_mu carries the shift of cubic_P, which
  // tile_N does not.
  static_assert(CORR, "k_tile runs the correction form only");
  pdl_enter();
  extern __shared__ __align__(16) unsigned char tile_smem[];
  const int SW = kTileW + 2 * halo, SH = kTileH + 2 * halo, SN = SW * SH;
  TileView<T, CORR> V;
  {
    T* base = reinterpret_cast<T*>(tile_smem);
    V.phi = base; V.mu = base + SN; V.p = base + 2 * SN; V.phim = base + 3 * SN; V.phis = base + 4 * SN;
    V.f1 = base + 5 * SN; V.f2 = base + 6 * SN; V.f3 = base + 7 * SN;
    V.phib = CORR ? base + 8 * SN : nullptr;
  }
  const int nx = L.nx, ny = L.ny;
  const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kTileH;  // tile origin (global)
  const int gx0 = tx0 - halo, gy0 = ty0 - halo;                      // shared-memory origin (global)

  // load the tile and its halo (cells outside the domain are never read)
  for (int s = threadIdx.x; s < SN; s += blockDim.x) {
    int sy = s / SW, sx = s - sy * SW;
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
    x1 = min(tx0 + kTileW + g, nx);
    y0 = max(ty0 - g, 0);
    y1 = min(ty0 + kTileH + g, ny);
  };

  if (rhs) {  // f += N(R u) wherever pass 1 needs f
    int x0, x1, y0, y1;
    region(halo - 1, x0, x1, y0, y1);
    const int w = x1 - x0, total = w * (y1 - y0);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int j = y0 + t / w, i = x0 + t % w;
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
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int j = y0 + t / hw;
      int i = x0 + 2 * (t % hw);
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
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int j = y0 + t / w, i = x0 + t % w;
      int s = (i - gx0) + SW * (j - gy0), c = i + nx * j;
      L.phi[c] = V.phi[s];
      L.mu[c] = V.mu[s];
      L.p[c] = V.p[s];
      if (rhs) {
        L.fphi[c] = V.f1[s];
        L.fmu[c] = V.f2[s];
        L.fp[c] = V.f3[s];
      }
    }
  }

  if (restrict_out) {  // residual on the tile and its restriction (coarse cell per thread)
    const int cw = kTileW / 2, chh = kTileH / 2;
    for (int t = threadIdx.x; t < cw * chh; t += blockDim.x) {
      const int I = (tx0 >> 1) + t % cw, J = (ty0 >> 1) + t / cw;
      if (I >= Cl.nx || J >= Cl.ny) continue;
      T r1 = 0, r2 = 0, r3 = 0, a = 0, b = 0, d = 0, e = 0;
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * J + dj;
          const int s = (i - gx0) + SW * (j - gy0);
          LocalCoef<T> C;
          local_coef(V.phis, s, SW, i, j, nx, ny, L, K, C);
          T n1, n2, n3;
          tile_N<T, CORR>(V, s, SW, i, j, nx, ny, L, K, C, n1, n2, n3);
          r1 += V.f1[s] - n1;
          r2 += V.f2[s] - n2;
          r3 += V.f3[s] - n3;
          a += V.phi[s];
          b += V.mu[s];
          d += V.p[s];
          if (CORR) e += V.phib[s];
        }
      const int q = I + Cl.nx * J;
      Cl.fphi[q] = T(0.25) * r1;
      Cl.fmu[q] = T(0.25) * r2;
      Cl.fp[q] = T(0.25) * r3;
      Cl.phi[q] = Cl.phi0[q] = T(0.25) * a;
      Cl.mu[q] = Cl.mu0[q] = T(0.25) * b;
      Cl.p[q] = Cl.p0[q] = T(0.25) * d;
      if (CORR) Cl.phib[q] = T(0.25) * e;
    }
  }
}

}  // namespace chhs_dev
