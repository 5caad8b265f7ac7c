// chhs_norm_df.cuh -- the mixed-precision form's defect-correction residual
// f - N(u) of the double-precision iterate, evaluated in double-single
// arithmetic (chhs_df64.cuh) on the single-precision pipes.
//
// Same outputs as k_norm_mixed: the stopping norm and the pointwise residual
// (the loop decision of the step graph), the mean of p, and the next inner
// solve's right-hand side (r rounded to single precision, e = 0,
// phi_b = phi cut to single precision).  The residual is formed in the
// difference form of Eqs. 2.5-2.7,
//   N1 = phi - s/h^2 sum_f [M_f (mu_e - mu_c) + a_f (p_e - p_c)]
//   N2 = mu + (3/4) eps^2/h^2 sum_f (phi_e - phi_c) - phi (phi^2 + phi phi^m + (phi^m)^2)/4
//   N3 = -1/h^2 sum_f [(p_e - p_c) + gamma a_f (mu_e - mu_c)]
// (N2 and f_mu carry the same constant shift (phi^m)^3/4 as the
// double-precision kernels, see cubic_P), with every double input split
// into hi + lo and every operation a double-single one: the residual is
// exact to ~1e-14 relative to the terms, far below the 1e-10 stopping
// tolerance, at a quarter of the issue slots of double precision on GB300.
//
// Each block takes a tile of 32 x 8 cells of one z-plane: the double state
// (phi, mu, p) and the +x/+y face coefficients of the tile and its one-cell
// ring are split once into shared memory; z-neighbours (3D) are split where
// they are read.
#pragma once
#include "chhs_df64.cuh"
#include "chhs_kernels.cuh"

namespace chhs_dev {

constexpr int kNdfTX = 32, kNdfTY = 8;  // 256 threads, one cell each
constexpr int kNdfSW = kNdfTX + 2, kNdfSH = kNdfTY + 2, kNdfSN = kNdfSW * kNdfSH;

// Blocks of the double-single norm on an nx x ny x nz grid.
__host__ __device__ inline int ndf_blocks_x(int nx) { return (nx + kNdfTX - 1) / kNdfTX; }
__host__ __device__ inline int ndf_blocks_y(int ny) { return (ny + kNdfTY - 1) / kNdfTY; }
__host__ __device__ inline long long ndf_blocks(int nx, int ny, int nz) {
  return (long long)ndf_blocks_x(nx) * ndf_blocks_y(ny) * nz;
}

// The level's scalar coefficients as double-single numbers (host-split).
struct DfCoefs {
  df64 sih2, ih2, e34ih2, gamma;
  float s;
};

// Block sums: thread 0 returns the sum of squares, the double-single sum of
// p and the maximum.
__device__ __forceinline__ void ndf_block_reduce(float& sq, df64& ps, float& mx) {
  __shared__ float s_sq[kNdfTX * kNdfTY / 32], s_mx[kNdfTX * kNdfTY / 32];
  __shared__ df64 s_ps[kNdfTX * kNdfTY / 32];
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_down_sync(0xffffffffu, sq, o);
    mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    const df64 other{__shfl_down_sync(0xffffffffu, ps.hi, o), __shfl_down_sync(0xffffffffu, ps.lo, o)};
    ps = df_add(ps, other);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_sq[wid] = sq;
    s_mx[wid] = mx;
    s_ps[wid] = ps;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      sq += s_sq[w];
      mx = fmaxf(mx, s_mx[w]);
      ps = df_add(ps, s_ps[w]);
    }
  }
  __syncthreads();
}

// The double-precision pipe and the single-precision/integer pipes work at
// the same time: a share of the blocks (f64_per8 of every 8) evaluates its
// tile's residual with double-precision instructions (eval_N), the others in
// double-single arithmetic; on one SM the former wait on the FP64 pipe while
// the latter fill the issue slots.  Both write the same outputs, and the
// residual is exact to far below the stopping tolerance either way.
//
// bx: the block's index among the run's nbx blocks (x-tiles fastest, then
// y-tiles, then z-planes).  Returns true in the run's last block (which took
// the loop decision).
template <int DIM>
__device__ __forceinline__ bool norm_mixed_df_body(int bx, int nbx, const Level<double>& L, const DfCoefs& K,
                                                   const Coefs<double>& K64, int f64_per8, const Level<float>& G,
                                                   double* partials, DevState* st, cudaGraphConditionalHandle cond,
                                                   int mode, int use_cond) {
  __shared__ df64 sP[kNdfSN], sU[kNdfSN], sQ[kNdfSN], sAx[kNdfSN], sMx[kNdfSN], sAy[kNdfSN], sMy[kNdfSN];
  __shared__ bool last;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int gx = ndf_blocks_x(nx), gy = ndf_blocks_y(ny);
  const int tx_blk = bx % gx;
  const int rest = bx / gx;
  const int ty_blk = rest % gy, k = rest / gy;
  const int x0 = tx_blk * kNdfTX, y0 = ty_blk * kNdfTY;
  const int sz = nx * ny;
  if ((bx & 7) < f64_per8) {  // this tile in double precision
    const int tx = threadIdx.x % kNdfTX, ty = threadIdx.x / kNdfTX;
    const int i = x0 + tx, j = y0 + ty;
    float sq = 0.f, mx = 0.f;
    df64 ps{0.f, 0.f};
    if (i < nx && j < ny) {
      const int c = i + nx * j + sz * k;
      double n1, n2, n3;
      eval_N<double, DIM, false>(L, K64, L.phi, L.mu, L.p, c, i, j, k, n1, n2, n3);
      const double r1 = L.fphi[c] - n1, r2 = L.fmu[c] - n2, r3 = L.fp[c] - n3;
      const float r1f = f64_to_f32_rz(r1), r2f = f64_to_f32_rz(r2), r3f = f64_to_f32_rz(r3);
      const float r3s = K.s * r3f;
      sq = r1f * r1f + r2f * r2f + r3s * r3s;
      mx = fmaxf(fmaxf(fabsf(r1f), fabsf(r2f)), fabsf(r3s));
      const double pc = L.p[c];
      ps = df_split(pc);
      G.fphi[c] = r1f;
      G.fmu[c] = r2f;
      G.fp[c] = r3f;
      G.phi[c] = 0.f;
      G.mu[c] = 0.f;
      G.p[c] = 0.f;
      G.phib[c] = f64_to_f32_rz(L.phi[c]);
    }
    ndf_block_reduce(sq, ps, mx);
    if (threadIdx.x == 0) {
      partials[3 * bx] = (double)sq;
      partials[3 * bx + 1] = df_to_double(ps);
      partials[3 * bx + 2] = (double)mx;
      __threadfence();
      last = atomicAdd(&st->ticket, 1u) == nbx - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    norm_finish(partials, nbx, L.ncell, st, cond, mode, use_cond);
    return true;
  }
  // the tile and its ring, split once
  for (int q = threadIdx.x; q < kNdfSN; q += blockDim.x) {
    const int qy = q / kNdfSW, qx = q - qy * kNdfSW;
    const int i = x0 - 1 + qx, j = y0 - 1 + qy;
    if (i < 0 || j < 0 || i >= nx || j >= ny) continue;
    const int c = i + nx * j + sz * k;
    sP[q] = df_split(L.phi[c]);
    sU[q] = df_split(L.mu[c]);
    sQ[q] = df_split(L.p[c]);
    sAx[q] = df_split(L.ax[c]);
    sMx[q] = df_split(L.Mx[c]);
    sAy[q] = df_split(L.ay[c]);
    sMy[q] = df_split(L.My[c]);
  }
  __syncthreads();
  const int tx = threadIdx.x % kNdfTX, ty = threadIdx.x / kNdfTX;
  const int i = x0 + tx, j = y0 + ty;
  float sq = 0.f, mx = 0.f;
  df64 ps{0.f, 0.f};
  if (i < nx && j < ny) {
    const int c = i + nx * j + sz * k;
    const int s = (tx + 1) + kNdfSW * (ty + 1);
    const df64 phic = sP[s], muc = sU[s], pc = sQ[s];
    df64 S1{0.f, 0.f}, Sa{0.f, 0.f}, Sp{0.f, 0.f}, Sphi{0.f, 0.f};
    auto face = [&](df64 phe, df64 mue, df64 pe, df64 a, df64 M) {
      const df64 dmu = df_sub(mue, muc), dp = df_sub(pe, pc), dphi = df_sub(phe, phic);
      S1 = df_add(S1, df_add(df_mul(M, dmu), df_mul(a, dp)));
      Sa = df_add(Sa, df_mul(a, dmu));
      Sp = df_add(Sp, dp);
      Sphi = df_add(Sphi, dphi);
    };
    if (i > 0) face(sP[s - 1], sU[s - 1], sQ[s - 1], sAx[s - 1], sMx[s - 1]);
    if (i + 1 < nx) face(sP[s + 1], sU[s + 1], sQ[s + 1], sAx[s], sMx[s]);
    if (j > 0) face(sP[s - kNdfSW], sU[s - kNdfSW], sQ[s - kNdfSW], sAy[s - kNdfSW], sMy[s - kNdfSW]);
    if (j + 1 < ny) face(sP[s + kNdfSW], sU[s + kNdfSW], sQ[s + kNdfSW], sAy[s], sMy[s]);
    if (DIM == 3) {
      if (k > 0) {
        const int e = c - sz;
        face(df_split(L.phi[e]), df_split(L.mu[e]), df_split(L.p[e]), df_split(L.az[e]), df_split(L.Mz[e]));
      }
      if (k + 1 < nz) {
        const int e = c + sz;
        face(df_split(L.phi[e]), df_split(L.mu[e]), df_split(L.p[e]), df_split(L.az[c]), df_split(L.Mz[c]));
      }
    }
    const df64 pm = df_split(L.phim[c]);
    // N1, N3 and the shifted N2 (see above)
    const df64 n1 = df_sub(phic, df_mul(K.sih2, S1));
    const df64 n3 = df_neg(df_mul(K.ih2, df_add(Sp, df_mul(K.gamma, Sa))));
    const df64 quad = df_add(df_mul(phic, df_add(phic, pm)), df_mul(pm, pm));
    const df64 cub = df_mul(df_mul(phic, quad), df64{0.25f, 0.f});
    const df64 n2 = df_sub(df_add(muc, df_mul(K.e34ih2, Sphi)), cub);
    const df64 r1 = df_sub(df_split(L.fphi[c]), n1);
    const df64 r2 = df_sub(df_split(L.fmu[c]), n2);
    const df64 r3 = df_sub(df_split(L.fp[c]), n3);
    const float r1f = df_to_float(r1), r2f = df_to_float(r2), r3f = df_to_float(r3);
    const float r3s = K.s * r3f;
    sq = r1f * r1f + r2f * r2f + r3s * r3s;
    mx = fmaxf(fmaxf(fabsf(r1f), fabsf(r2f)), fabsf(r3s));
    ps = pc;
    G.fphi[c] = r1f;
    G.fmu[c] = r2f;
    G.fp[c] = r3f;
    G.phi[c] = 0.f;
    G.mu[c] = 0.f;
    G.p[c] = 0.f;
    G.phib[c] = phic.hi;  // phi with its significand cut to 24 bits
  }
  ndf_block_reduce(sq, ps, mx);
  if (threadIdx.x == 0) {
    partials[3 * bx] = (double)sq;
    partials[3 * bx + 1] = df_to_double(ps);
    partials[3 * bx + 2] = (double)mx;
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
__global__ void __launch_bounds__(kNdfTX * kNdfTY) k_norm_mixed_df(const __grid_constant__ Level<double> L,
                                                                 DfCoefs K, Coefs<double> K64, int f64_per8,
                                                                 const __grid_constant__ Level<float> G,
                                                                 double* partials, DevState* st,
                                                                 cudaGraphConditionalHandle cond, int mode,
                                                                 int use_cond) {
  pdl_enter();
  norm_mixed_df_body<DIM>(blockIdx.x, gridDim.x, L, K, K64, f64_per8, G, partials, st, cond, mode, use_cond);
}

}  // namespace chhs_dev
