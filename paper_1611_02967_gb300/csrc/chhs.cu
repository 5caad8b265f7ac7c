// chhs.cu -- host side of the C ABI declared in include/chhs.h: argument
// checks, the device hierarchy in one arena, and the per-step CUDA graph.
//
// One time step is one CUDA graph launch:
//   setup (phi*, right-hand sides, initial guess)     Eq. 2.4 and 2.5-2.7
//   restrict phi^m, phi* to every coarse level
//   stopping norm -> while-loop condition
//   WHILE (norm > tol and V < max_v):                 Section 5 preamble
//       IF (inner >= 3) V-cycle; IF (inner >= 2) V-cycle;
//       V(nu1, nu2)-cycle; stopping norm -> conditions
//   mean of p; accept the step (rotate phi^m, phi^{m-1})
// The loop is a conditional graph node whose condition a device kernel sets,
// so a step needs no host round trip; the norm kernel also predicts how many
// V-cycles the next iteration runs (loop_decision).  chhs_step(n) launches
// the graph n times and reads the device status once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/chhs.h"
#include "chhs_kernels.cuh"
#include "chhs_tile.cuh"
#include "chhs_corr3.cuh"
#include "chhs_norm_df.cuh"
#include "chhs_batch.cuh"

using namespace chhs_dev;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int nblocks(int n) { return (n + kBlock - 1) / kBlock; }

struct Shape {
  int dim;
  int n[3];  // n[2] == 1 in 2D
};

// Level sizes: coarsen every direction by 2 while all stay even and >= coarsest.
std::vector<Shape> level_shapes(int dim, const int n[3], int coarsest) {
  std::vector<Shape> out;
  Shape s{dim, {n[0], n[1], dim == 3 ? n[2] : 1}};
  out.push_back(s);
  for (;;) {
    bool ok = true;
    for (int a = 0; a < dim; ++a)
      if (s.n[a] % 2 != 0 || s.n[a] / 2 < coarsest) ok = false;
    if (!ok) break;
    for (int a = 0; a < dim; ++a) s.n[a] /= 2;
    out.push_back(s);
  }
  return out;
}

// Per-level fields: phi mu p fphi fmu fp phim phis phi0 mu0 p0, ax ay Mx My,
// sM sa, cAe cC cGn cHn cQ cH (+ az Mz in 3D), in single precision also phi_b,
// and in 2D single precision (the tiled levels) a second (phi, mu, p) and the
// completed right-hand side.
constexpr int kBaseFields = 11;
int level_fields(int dim, bool single) {
  return kBaseFields + (dim == 3 ? 14 : 12) + (single ? 1 + (dim == 2 ? 6 : 0) : 0);
}

// The mixed form's residual kernel: of every 8 tiles, this many are evaluated
// with double-precision instructions and the rest in double-single
// arithmetic, so that both kinds of pipes are busy (chhs_norm_df.cuh).
constexpr int kNormF64Per8 = 3;

// Tiles of the 2D single-precision levels: a level of at least
// kLargeTileCells cells takes chhs_tuning's tile_* (default 32 x 32 cells on
// 512 threads), a smaller one small_tile_* (default 16 x 8 on 256: four times
// the blocks on the small, latency-bound levels).  On the 512^2 mixed step
// 16 x 8 below the finest level measured 4% faster than 32 x 16 there, and
// 32 x 32 on levels of 256 x 512 cells and more took the batched
// configuration's large runs from 6.3e8 to 7.2e8 cell-steps/s.
constexpr int kLargeTileW = 32, kLargeTileH = 32, kLargeTileThreads = 512;
constexpr int kSmallTileW = 16, kSmallTileH = 8, kSmallTileThreads = 256;
constexpr int kLargeTileCells = 512 * 256;

// Levels with at most this many cells run inside the one-block tail kernel.
// In double precision one SM does 2 FMA per clock and a single warp's
// dependent FP64 chain is slow, so only the tiniest levels (8 x 8, 4 x 4 x 4)
// go there; in single precision (64x the rate) levels up to 32 x 32 do.
constexpr int kTailCellsF64 = 64;
constexpr int kTailCellsF32 = 1024;

// Double-precision levels with at most this many threads per colour pass
// (one per cell of the colour) use the split update (k_smooth_split): up to
// 128 x 128 in 2D, where a pass has at most one warp per sub-partition's
// worth of groups.
constexpr int kSplitThreads = 8192;

struct Layout {
  std::vector<Shape> shapes;
  size_t state_off, partial_off, phimm1_off;
  int nlev64;                       // double-precision levels (all, or the finest only when mixed)
  std::vector<size_t> level_off;    // start of each double-precision level's arrays
  std::vector<size_t> level32_off;  // start of each single-precision level's arrays (mixed only)
  size_t total;
  int nparts;  // partial-sum slots (blocks of the finest grid)
};

Layout make_layout(int dim, const int n[3], int coarsest, int precision) {
  Layout L;
  L.shapes = level_shapes(dim, n, coarsest);
  size_t off = 0;
  L.state_off = off;
  off += align_up(sizeof(DevState));
  int nf = L.shapes[0].n[0] * L.shapes[0].n[1] * L.shapes[0].n[2];
  // partial-sum slots: six per 256-cell block (the reductions), and three per
  // block of the double-single norm (tiles of 32 x 8 cells)
  L.nparts = (int)std::max<long long>(nblocks(nf),
                                      (ndf_blocks(L.shapes[0].n[0], L.shapes[0].n[1], L.shapes[0].n[2]) + 1) / 2);
  L.partial_off = off;
  off += align_up(sizeof(double) * 6 * (size_t)L.nparts);
  L.phimm1_off = off;
  off += align_up(sizeof(double) * (size_t)nf);
  L.nlev64 = precision == 1 ? 1 : (int)L.shapes.size();
  for (int l = 0; l < L.nlev64; ++l) {
    const Shape& s = L.shapes[l];
    size_t nc = (size_t)s.n[0] * s.n[1] * s.n[2];
    L.level_off.push_back(off);
    off += level_fields(dim, false) * align_up(sizeof(double) * nc);
  }
  if (precision == 1)
    for (const Shape& s : L.shapes) {
      size_t nc = (size_t)s.n[0] * s.n[1] * s.n[2];
      L.level32_off.push_back(off);
      off += level_fields(dim, true) * align_up(sizeof(float) * nc);
    }
  L.total = off;
  return L;
}

// coarsest >= 2: a level of one cell per direction has no interior face, so
// its Newton diagonal and the pressure row have nothing to work with (the
// pressure problem is singular and the face count 0 has no inverse).
bool valid_opts(const chhs_opts& o) {
  return o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 >= 1 && o.max_v >= 1 && o.coarsest >= 2 &&
         o.tol > 0 && (o.precision == 0 || o.precision == 1) && o.max_factor >= 0 &&
         (o.coarsest_f64 == 0 || o.coarsest_f64 == 1) && (o.f64_residual == 0 || o.f64_residual == 1) &&
         o.max_inner >= 1 && o.max_inner <= kMaxInner;
}

bool valid_problem(int dim, const int n[3], double h, double eps, double gamma, double dt) {
  if (dim != 2 && dim != 3) return false;
  if (!n) return false;
  long long cells = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 2 || n[a] > (1 << 20)) return false;
    cells *= n[a];
  }
  if (cells > (1LL << 31) / 8) return false;  // 32-bit cell indices with headroom
  return h > 0 && eps > 0 && dt > 0 && gamma >= 0 && std::isfinite(h) && std::isfinite(eps) &&
         std::isfinite(dt) && std::isfinite(gamma);
}

// Event pairs around launches while chhs_profile_step runs.
struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  std::vector<double> units;
  size_t used = 0;
  cudaEvent_t next() {
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    return ev[used++];
  }
  ~Prof() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

}  // namespace

struct chhs {
  int dim = 2;
  int n[3] = {1, 1, 1};
  double h = 0, eps = 0, gamma = 0, dt = 0;
  chhs_opts opts{};
  Layout layout;
  char* arena = nullptr;
  bool own_arena = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Level<double>> lev;   // double precision: all levels, or the finest only when mixed
  std::vector<Level<float>> lev32;  // single-precision correction hierarchy (mixed precision)
  int tail_start = 0;               // first level run by the one-block tail kernel
  // launch shapes (defaults above; chhs_autotune may change them): levels of at
  // most tail_cells cells go to the tail, double-precision levels of at most
  // split_threads threads per colour pass use the split update, tiles run
  // tile_threads threads
  int tail_cells = 0, split_threads = kSplitThreads, tile_threads = kLargeTileThreads;
  int norm_blocks = 1;              // grid of the stopping-norm kernels (whole blocks per SM)
  int nu1c = 2, nu2c = 2;           // sweeps on the levels below the finest (chhs_autotune; opts by default)
  // tile interiors of the 2D single-precision levels of at least
  // kLargeTileCells cells (tile_*) and of the smaller ones (stile_*, with its
  // block size; chhs_autotune)
  int tile_w = kLargeTileW, tile_h = kLargeTileH;
  int stile_w = kSmallTileW, stile_h = kSmallTileH, stile_threads = kSmallTileThreads;
  int norm_f64_per8 = kNormF64Per8;      // blocks of 8 whose residual runs on the FP64 pipe (mixed form)
  int quad_passes = 1;              // 3D mixed form: x-quad colour passes where nx % 4 == 0 (k_smooth_c4)
  Tail<double> tail{};              // its levels (double-precision V-cycles)
  Tail<float> tail32{};             // (single-precision inner V-cycles)
  double* phimm1 = nullptr;
  DevState* st = nullptr;
  double* partials = nullptr;
  DevState* host_st = nullptr;  // pinned mirror
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches_per_v = 0, launches_per_step = 0;
  bool vc_update = true;  // while enqueueing: this V-cycle ends with the update u <- u + e (mixed form)
  bool pending = false;  // steps enqueued by chhs_step_async since the last chhs_wait
  int* counter = nullptr;  // counts launches while the graph is captured
  Prof* prof = nullptr;  // per-launch events while profiling
  bool batch_member = false;  // a run of a chhs_batch: stepped by the batch's graph, freed by the batch
  std::string err;
  int ncell() const { return n[0] * n[1] * n[2]; }
};

namespace {

void destroy_handle(chhs_t* run);

chhs_status fail(chhs_t* r, chhs_status s, const std::string& msg) {
  if (r) r->err = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(run, CHHS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Every kernel of the solver goes through here: counted while the graph is
// captured, bracketed by events while profiling.
template <class F>
void launch(chhs_t* run, cudaStream_t s, int kind, double units, F&& f) {
  if (run->counter) ++*run->counter;
  if (run->prof) {
    cudaEvent_t a = run->prof->next(), b = run->prof->next();
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    run->prof->kind.push_back(kind);
    run->prof->units.push_back(units);
  } else {
    f();
  }
}

// Launches of a step's kernels allow programmatic dependent launch: the next
// kernel may be scheduled while the previous one drains; each kernel waits
// for its predecessor's completion itself (pdl_enter).  Measured on the
// 512 x 512 workload: 2-4% per step.
template <typename... KArgs, typename... Args>
void pdl_smem(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
void pdl_grid(void (*kernel)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
void pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  pdl_smem(kernel, grid, block, 0, s, args...);
}

// Cells of colour 0 ((i+j+k) even) in a box whose corner cell is even.
template <typename T>
double colour_cells(const Level<T>& L, int colour) {
  double n = L.ncell;
  bool odd = (L.ncell & 1) != 0;
  return colour == 0 ? (odd ? (n + 1) / 2 : n / 2) : (odd ? (n - 1) / 2 : n / 2);
}

template <int DIM>
struct Enqueue {
  template <typename T>
  static Coefs<T> coefs(const chhs_t* run) {
    return Coefs<T>{T(run->dt), T(run->gamma), T(0.75 * run->eps * run->eps)};
  }

  // Sweeps before and after the coarse-grid correction on level l: the
  // options' counts on the finest level, the handle's coarse counts below.
  static int nu_pre(const chhs_t* run, int l) { return l == 0 ? run->opts.nu1 : run->nu1c; }
  static int nu_post(const chhs_t* run, int l) { return l == 0 ? run->opts.nu2 : run->nu2c; }

  // sweeps red-black sweeps; with rhs the first one also completes the FAS
  // right-hand side of this (coarse) level.
  template <typename T, bool CORR>
  static void smooth(chhs_t* run, cudaStream_t s, const Level<T>& L, int sweeps, bool rhs) {
    const Coefs<T> K = coefs<T>(run);
    const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
    const int blocks = (threads + kSmoothBlock - 1) / kSmoothBlock;
    // small double-precision levels: each cell's update split over three warps
    const bool split = std::is_same<T, double>::value && !CORR && threads <= run->split_threads &&
                       L.ncell != run->ncell();
    for (int it = 0; it < sweeps; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        const int with_rhs = (rhs && it == 0) ? 1 : 0;
        const int kind = L.ncell == run->ncell() ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH;
        launch(run, s, kind, colour_cells(L, colour), [&] {
          if constexpr (std::is_same<T, double>::value && !CORR) {
            if (split) {
              pdl(k_smooth_split<DIM>, (threads + 31) / 32, 96, s, L, K, colour, with_rhs);
              return;
            }
          }
          pdl(k_smooth<T, DIM, CORR>, blocks, kSmoothBlock, s, L, K, colour, with_rhs);
        });
      }
  }

  // One FAS V(nu1, nu2)-cycle from level l down, on a hierarchy of either precision.
  template <typename T, bool CORR>
  static void vcycle(chhs_t* run, cudaStream_t s, const std::vector<Level<T>>& lev, const Tail<T>& tail,
                     int l) {
    const Coefs<T> K = coefs<T>(run);
    const Level<T>& L = lev[l];
    if (l == run->tail_start) {
      const size_t smem = tail_bytes<T, CORR>(tail);
      launch(run, s, CHHS_K_COARSEST, 1.0, [&] {
        pdl_smem(k_tail<T, DIM, CORR>, 1, kTailThreads, smem, s, tail, K);
      });
      return;
    }
    const Level<T>& C = lev[l + 1];
    const bool rhs = l > 0;
    if constexpr (use_tiles<T>()) {
      // 2D single precision: pre-smoothing (+ right-hand side) + residual +
      // restriction in one tiled launch, prolongation + post-smoothing in another
      const bool large = L.ncell >= kLargeTileCells;
      const int tw = large ? run->tile_w : run->stile_w, th = large ? run->tile_h : run->stile_h;
      const int tt = large ? run->tile_threads : run->stile_threads;
      const dim3 grid((L.nx + tw - 1) / tw, (L.ny + th - 1) / th);
      const int nf = tile_nfields<CORR>();
      const int np1 = 2 * nu_pre(run, l), np2 = 2 * nu_post(run, l);
      // the pre-smoothing launch writes the second copy of the state (and the
      // completed right-hand side), the post-smoothing launch reads them and
      // writes the state back: no launch writes what its own tiles read
      const TileOut<T> to_copy{L.phi2, L.mu2, L.p2, L.fc1, L.fc2, L.fc3, nullptr, nullptr, nullptr};
      Level<T> Lb = L;
      Lb.phi = L.phi2;
      Lb.mu = L.mu2;
      Lb.p = L.p2;
      if (rhs) {
        Lb.fphi = L.fc1;
        Lb.fmu = L.fc2;
        Lb.fp = L.fc3;
      }
      TileOut<T> to_state{L.phi, L.mu, L.p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
      if (l == 0 && fused_update(run) && run->vc_update) {  // the finished correction goes straight into u
        to_state.phi64 = run->lev[0].phi;
        to_state.mu64 = run->lev[0].mu;
        to_state.p64 = run->lev[0].p;
      }
      launch(run, s, l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, (double)L.ncell * nu_pre(run, l), [&] {
        pdl_grid(k_tile<T, CORR>, grid, tt, tile_smem_bytes(np1 + 1, nf, sizeof(T), tw, th), s, L, C,
                 K, np1, np1 + 1, rhs ? 1 : 0, 0, 1, to_copy, (const int*)nullptr, tw, th);
      });
      vcycle<T, CORR>(run, s, lev, tail, l + 1);
      launch(run, s, l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, (double)L.ncell * nu_post(run, l), [&] {
        pdl_grid(k_tile<T, CORR>, grid, tt, tile_smem_bytes(np2, nf, sizeof(T), tw, th), s, Lb, C, K,
                 np2, np2, 0, 1, 0, to_state, (const int*)nullptr, tw, th);
      });
      return;
    }
    if (rhs && nu_pre(run, l) == 0)
      launch(run, s, CHHS_K_COARSE_RHS, L.ncell, [&] {
        pdl(k_coarse_rhs<T, DIM, CORR>, nblocks(L.ncell), kBlock, s, L, K);
      });
    if constexpr (recompute_coefs<T, CORR>()) {
      corr_vcycle_level(run, s, lev, tail, l);
      return;
    }
    smooth<T, CORR>(run, s, L, nu_pre(run, l), rhs && nu_pre(run, l) > 0);
    constexpr int TX = DIM == 3 ? 8 : 16;
    const long long tiles = (long long)((L.nx + TX - 1) / TX) * (L.ny / 2) * (DIM == 3 ? L.nz / 2 : 1);
    const int rblocks = (int)((tiles * 32 + kBlock - 1) / kBlock);
    launch(run, s, CHHS_K_RESTRICT, L.ncell, [&] {
      if constexpr (std::is_same<T, double>::value && !CORR) {
        if (L.ncell <= 2 * run->split_threads && l > 0) {  // small level: the three rows on three warps
          pdl(k_residual_restrict_split<DIM>, (int)tiles, 96, s, L, C, K);
          return;
        }
      }
      pdl(k_residual_restrict<T, DIM, CORR>, rblocks, kBlock, s, L, C, K);
    });
    vcycle<T, CORR>(run, s, lev, tail, l + 1);
    launch(run, s, CHHS_K_PROLONG, L.ncell, [&] {
      pdl(k_prolong<T, DIM>, nblocks(L.ncell), kBlock, s, L, C);
    });
    smooth<T, CORR>(run, s, L, nu_post(run, l), false);
  }

  // 3D single-precision (correction-form) levels above the tail: colour
  // passes with the coefficients recomputed from phi* (k_smooth_c), the
  // prolongation folded into the first post-smoothing sweep and, on the
  // finest level, the update u <- u + e into the last pass.
  template <typename T, bool CORR>
  static constexpr bool recompute_coefs() { return DIM == 3 && std::is_same<T, float>::value && CORR; }

  static void corr_vcycle_level(chhs_t* run, cudaStream_t s, const std::vector<Level<float>>& lev,
                                const Tail<float>& tail, int l) {
    const Coefs<float> K = coefs<float>(run);
    const Level<float>& L = lev[l];
    const Level<float>& C = lev[l + 1];
    const bool rhs = l > 0;
    const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
    const int blocks = (threads + kSmoothBlock - 1) / kSmoothBlock;
    const int kind = l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH;
    const Level<double> none{};
    const int nu1 = nu_pre(run, l), nu2 = nu_post(run, l);
    // one colour pass: x-quads (k_smooth_c4, the same results bit for bit)
    // where the rows split into whole quads, else one cell per thread
    auto pass = [&](int colour, int with_rhs, int pro, const Level<double>& U) {
      if constexpr (DIM == 3) {
        if (quad_level(run, L)) {
          const dim3 qg = quad_grid(L.nx, L.ny, L.nz);
          const int tl = quad_tile(L.nx);
          if (with_rhs)
            pdl_grid(k_smooth_c4<1, 0>, qg, kSmoothBlock, 0, s, L, C, K, colour, U, tl);
          else if (pro == 1)
            pdl_grid(k_smooth_c4<0, 1>, qg, kSmoothBlock, 0, s, L, C, K, colour, U, tl);
          else if (pro == 2)
            pdl_grid(k_smooth_c4<0, 2>, qg, kSmoothBlock, 0, s, L, C, K, colour, U, tl);
          else
            pdl_grid(k_smooth_c4<0, 0>, qg, kSmoothBlock, 0, s, L, C, K, colour, U, tl);
          return;
        }
      }
      pdl(k_smooth_c<DIM>, blocks, kSmoothBlock, s, L, C, K, colour, with_rhs, pro, U);
    };
    for (int it = 0; it < nu1; ++it)
      for (int colour = 0; colour < 2; ++colour)
        launch(run, s, kind, colour_cells(L, colour), [&] { pass(colour, (rhs && it == 0) ? 1 : 0, 0, none); });
    const long long warps = rr_c_warps(DIM, L.nx, L.ny, L.nz);
    const int rblocks = (int)((warps * 32 + kBlock - 1) / kBlock);
    launch(run, s, CHHS_K_RESTRICT, L.ncell, [&] {
      pdl(k_residual_restrict_c<DIM>, rblocks, kBlock, s, L, C, K);
    });
    vcycle<float, true>(run, s, lev, tail, l + 1);
    if (nu2 == 0) {
      launch(run, s, CHHS_K_PROLONG, L.ncell, [&] {
        pdl(k_prolong<float, DIM>, nblocks(L.ncell), kBlock, s, L, C);
      });
      return;
    }
    for (int it = 0; it < nu2; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        const int pro = it == 0 ? (colour == 0 ? 1 : 2) : 0;
        const bool upd = l == 0 && fused_update(run) && run->vc_update && it == nu2 - 1 && colour == 1;
        launch(run, s, kind, colour_cells(L, colour), [&] { pass(colour, 0, pro, upd ? run->lev[0] : none); });
      }
  }

  static bool mixed(const chhs_t* run) { return run->opts.precision == 1; }

  // A 3D single-precision level whose colour passes run as x-quads.
  static bool quad_level(const chhs_t* run, const Level<float>& L) {
    if (DIM != 3 || !run->quad_passes || L.nx % 4 != 0) return false;
    const dim3 g = quad_grid(L.nx, L.ny, L.nz);
    return g.y <= 65535 && g.z <= 65535;
  }

  // Mixed form whose finest level is not in the tail: the last smoothing
  // launch of a V-cycle performs the update u <- u + e (the 2D tile, or in 3D
  // the last colour pass when there is post-smoothing); k_mixed_update otherwise.
  static bool fused_update(const chhs_t* run) {
    return mixed(run) && run->tail_start > 0 && (DIM == 2 || run->opts.nu2 > 0);
  }

  // The fused tile kernels serve the 2D single-precision V-cycles.
  template <typename T>
  static constexpr bool use_tiles() { return DIM == 2 && std::is_same<T, float>::value; }

  template <typename T, bool CORR>
  static size_t tail_bytes(const Tail<T>& tail) {
    int nc[kTailMaxLevels];
    for (int l = 0; l < tail.n; ++l) nc[l] = tail.lev[l].ncell;
    return tail_smem_bytes<T, DIM, CORR>(nc, tail.n, tail.coarsest_f64);
  }

  // Opt the tail kernel in to the shared memory its levels need.
  template <typename T, bool CORR>
  // A grid that does not coarsen far enough leaves a coarsest level too large
  // for the one-block tail, and very long sweeps make the tiles' halos too
  // large: both are rejected as invalid arguments before any launch.
  static chhs_status prepare_tail(chhs_t* run, const Tail<T>& tail) {
    int dev = 0, optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    auto fits = [&](const void* fn, size_t dyn) {
      cudaFuncAttributes fa;
      return cudaFuncGetAttributes(&fa, fn) == cudaSuccess && dyn + fa.sharedSizeBytes <= (size_t)optin;
    };
    // the opt-in is per kernel and process-wide: only ever raise it, so that no
    // handle lowers it below what another handle's graph launches need
    auto raise_to = [&](const void* fn, size_t dyn) -> cudaError_t {
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, fn);
      if (e != cudaSuccess || (size_t)fa.maxDynamicSharedSizeBytes >= dyn) return e;
      return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    };
    const size_t smem = tail_bytes<T, CORR>(tail);
    const void* ktail = reinterpret_cast<const void*>(k_tail<T, DIM, CORR>);
    if (!fits(ktail, smem))
      return fail(run, CHHS_ERR_INVALID_ARG,
                  "the grid does not coarsen to a coarsest level small enough for the one-block solve");
    CU(raise_to(ktail, smem));
    if constexpr (use_tiles<T>()) {
      const int halo = 2 * std::max(std::max(run->opts.nu1, run->opts.nu2), std::max(run->nu1c, run->nu2c)) + 1;
      const size_t tb = std::max(tile_smem_bytes(halo, tile_nfields<CORR>(), sizeof(T), run->tile_w, run->tile_h),
                                 tile_smem_bytes(halo, tile_nfields<CORR>(), sizeof(T), run->stile_w, run->stile_h));
      const void* ktile = reinterpret_cast<const void*>(k_tile<T, CORR>);
      if (!fits(ktile, tb))
        return fail(run, CHHS_ERR_INVALID_ARG, "nu1/nu2 too large for the single-precision tiles");
      CU(raise_to(ktile, tb));
    }
    return CHHS_OK;
  }

  // The finest level's scalars for the double-single residual.
  static DfCoefs df_coefs(const chhs_t* run) {
    const Level<double>& L = run->lev[0];
    return DfCoefs{df_from_double_host(L.sih2), df_from_double_host(L.ih2), df_from_double_host(L.e34ih2),
                   df_from_double_host(run->gamma), (float)run->dt};
  }

  // The stopping norm (and, when mixed, the next inner solve's right-hand side).
  static void norm(chhs_t* run, cudaStream_t s, cudaGraphConditionalHandle cond, int mode, int use_cond) {
    const Coefs<double> K = coefs<double>(run);
    const Level<double>& L = run->lev[0];
    const int nb = run->norm_blocks;
    launch(run, s, CHHS_K_NORM, L.ncell, [&] {
      if (mixed(run) && !run->opts.f64_residual)
        pdl(k_norm_mixed_df<DIM>, (int)ndf_blocks(L.nx, L.ny, L.nz), kNdfTX * kNdfTY, s, L, df_coefs(run), K,
            run->norm_f64_per8, run->lev32[0], run->partials, run->st, cond, mode, use_cond);
      else if (mixed(run))
        pdl(k_norm_mixed<DIM>, nb, kBlock, s, L, K, run->lev32[0], run->partials, run->st, cond, mode, use_cond);
      else
        pdl(k_norm<double, DIM>, nb, kBlock, s, L, K, run->partials, run->st, cond, mode, use_cond);
    });
  }

  // One V-cycle of the step's loop: a double-precision V-cycle, or a
  // single-precision correction V-cycle, followed (update) by the
  // double-precision update u <- u + e.  An iteration of the loop runs
  // DevState::inner V-cycles, the update after the last only (the ones before
  // continue the same correction equation from the correction they leave),
  // then the stopping norm.
  static void vcycle_step(chhs_t* run, cudaStream_t s, bool update) {
    if (mixed(run)) {
      run->vc_update = update;
      vcycle<float, true>(run, s, run->lev32, run->tail32, 0);
      run->vc_update = true;
      const Level<double>& L = run->lev[0];
      if (update && !fused_update(run))
        launch(run, s, CHHS_K_FRAME, 1.0, [&] {
          pdl(k_mixed_update, nblocks(L.ncell), kBlock, s, L, run->lev32[0]);
        });
    } else {
      vcycle<double, false>(run, s, run->lev, run->tail, 0);
    }
  }

  // The step's set-up: phi*, f, the initial guess and the finest level's
  // coefficients (frame_setup), then the coarser levels' coefficients
  // (frame_coefs), which only the V-cycles need: in the step graph they run
  // beside the initial stopping norm.
  static void frame_head(chhs_t* run, cudaStream_t s) {
    frame_setup(run, s);
    frame_coefs(run, s);
  }

  static void frame_setup(chhs_t* run, cudaStream_t s) {
    const Level<double>& F = run->lev[0];
    const Coefs<double> K = coefs<double>(run);
    const std::vector<Level<double>>& D = run->lev;
    const int nd = (int)D.size();
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      pdl(k_setup_coef<DIM>, nblocks(F.ncell), kBlock, s, F, run->phimm1, run->eps * run->eps, run->st, K,
          nd > 1 ? D[1] : D[0], nd > 1 ? 1 : 0);
    });
  }

  static void frame_coefs(chhs_t* run, cudaStream_t s) {
    const Level<double>& F = run->lev[0];
    const Coefs<double> K = coefs<double>(run);
    const std::vector<Level<double>>& D = run->lev;
    const int nd = (int)D.size();
    for (int l = 1; l < nd; ++l)
      launch(run, s, CHHS_K_FRAME, 1.0, [&] {
        pdl(k_coef_restrict<double, DIM>, nblocks(D[l].ncell), kBlock, s, D[l], K, l + 1 < nd ? D[l + 1] : D[l],
            l + 1 < nd ? 1 : 0);
      });
    if (!mixed(run)) return;
    const std::vector<Level<float>>& G = run->lev32;
    const int ng = (int)G.size();
    const Coefs<float> K32 = coefs<float>(run);
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      pdl(k_coef_restrict_f32<DIM>, nblocks(F.ncell), kBlock, s, F, G[0], K32, ng > 1 ? G[1] : G[0],
          ng > 1 ? 1 : 0);
    });
    for (int l = 1; l < ng; ++l)
      launch(run, s, CHHS_K_FRAME, 1.0, [&] {
        pdl(k_coef_restrict<float, DIM>, nblocks(G[l].ncell), kBlock, s, G[l], K32, l + 1 < ng ? G[l + 1] : G[l],
            l + 1 < ng ? 1 : 0);
      });
  }

  static void frame_tail(chhs_t* run, cudaStream_t s) {
    const Level<double>& F = run->lev[0];
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      pdl(k_advance, nblocks(F.ncell), kBlock, s, F, run->phimm1, run->st);
    });
  }

  static chhs_status build_graph(chhs_t* run) {
    chhs_status ps = mixed(run) ? prepare_tail<float, true>(run, run->tail32) : prepare_tail<double, false>(run, run->tail);
    if (ps != CHHS_OK) return ps;
    // capture streams and fork/join events, released on every return path (a
    // capture that an error interrupted is ended and its graph dropped first)
    struct CaptureRes {
      cudaStream_t s[4] = {nullptr, nullptr, nullptr, nullptr};
      cudaEvent_t e[2] = {nullptr, nullptr};
      ~CaptureRes() {
        for (int q : {3, 1, 0}) {
          cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
          if (s[q] && cudaStreamIsCapturing(s[q], &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s[q], &g);
            if (q == 0 && g) cudaGraphDestroy(g);  // the body graph belongs to the step graph
          }
        }
        for (cudaEvent_t ev : e)
          if (ev) cudaEventDestroy(ev);
        for (cudaStream_t st : s)
          if (st) cudaStreamDestroy(st);
        cudaGetLastError();
      }
    } res;
    CU(cudaStreamCreateWithFlags(&res.s[0], cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&res.s[1], cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&res.s[2], cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&res.s[3], cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&res.e[0], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&res.e[1], cudaEventDisableTiming));
    cudaStream_t cs = res.s[0], cs2 = res.s[1], cs3 = res.s[2], cs4 = res.s[3];
    cudaEvent_t fork = res.e[0], join = res.e[1];
    int n_frame = 0, n_v = 0, n_other = 0;
    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    run->counter = &n_frame;
    frame_setup(run, cs);
    // the coarser levels' coefficients on a side branch, beside the initial norm
    CU(cudaEventRecord(fork, cs));
    CU(cudaStreamWaitEvent(cs3, fork, 0));
    frame_coefs(run, cs3);
    CU(cudaEventRecord(join, cs3));
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    CU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle cond;
    CU(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    norm(run, cs, cond, 0, 1);
    CU(cudaStreamWaitEvent(cs, join, 0));
    CU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp{};  // every other field zero
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    CU(cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp));
    CU(cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // the loop body: IF (inner >= 4) V-cycle; IF (inner >= 3) V-cycle; IF
    // (inner >= 2) V-cycle; the V-cycle with the update; the stopping norm,
    // which sets the loop condition and the IF conditions for the next
    // iteration
    const int n_if = std::min(run->opts.max_inner, kMaxInner) - 1;
    cudaGraphConditionalHandle cif[kMaxInner - 1] = {};
    for (int q = n_if - 1; q >= 0; --q) {
      cudaGraph_t bg = nullptr;
      CU(cudaStreamGetCaptureInfo(cs2, &cst, nullptr, &bg, &deps, nullptr, &ndeps));
      CU(cudaGraphConditionalHandleCreate(&cif[q], bg, 0, cudaGraphCondAssignDefault));
      cudaGraphNodeParams ip{};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = cif[q];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t ifn;
      CU(cudaGraphAddNode(&ifn, bg, deps, nullptr, ndeps, &ip));
      CU(cudaStreamUpdateCaptureDependencies(cs2, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
      cudaGraph_t ib = ip.conditional.phGraph_out[0];
      CU(cudaStreamBeginCaptureToGraph(cs4, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      run->counter = &n_other;
      vcycle_step(run, cs4, false);
      CU(cudaStreamEndCapture(cs4, &ib));
    }
    run->counter = &n_v;
    vcycle_step(run, cs2, true);
    run->counter = &n_other;
    norm(run, cs2, cond, 1, 1);
    CU(cudaStreamEndCapture(cs2, &body));
    run->counter = &n_frame;
    frame_tail(run, cs);
    run->counter = nullptr;
    CU(cudaStreamEndCapture(cs, &run->graph));
    CU(cudaGraphInstantiate(&run->exec, run->graph, 0));
    run->launches_per_v = n_v;
    run->launches_per_step = n_frame;
    // the IF nodes' handles, for the norm kernels that set them
    const int use_if = std::max(n_if, 0);
    CU(cudaMemcpyAsync(&run->st->use_if, &use_if, sizeof(int), cudaMemcpyHostToDevice, run->stream));
    CU(cudaMemcpyAsync(run->st->cond_if, cif, sizeof(cif), cudaMemcpyHostToDevice, run->stream));
    CU(cudaStreamSynchronize(run->stream));
    return CHHS_OK;
  }

  // One step launched kernel by kernel with events (see chhs_profile_step).
  static chhs_status profile_step(chhs_t* run) {
    cudaStream_t s = run->stream;
    frame_head(run, s);
    norm(run, s, 0, 0, 0);
    for (;;) {
      CU(cudaMemcpyAsync(run->host_st, run->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (!run->host_st->go) break;
      const int inner = std::max(1, run->host_st->inner);
      for (int q = 0; q < inner; ++q) vcycle_step(run, s, q == inner - 1);
      norm(run, s, 0, 1, 0);
    }
    frame_tail(run, s);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
    return CHHS_OK;
  }

  static chhs_status dissipation(chhs_t* run) {
    const int nb = nblocks(run->ncell());
    k_dissip_partial<DIM><<<nb, kBlock, 0, run->stream>>>(run->lev[0], run->gamma, 1.0 / run->h, run->partials);
    k_dissip_finish<<<1, 32, 0, run->stream>>>(run->partials, nb, run->st);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(run->host_st, run->st, sizeof(DevState), cudaMemcpyDeviceToHost, run->stream));
    CU(cudaStreamSynchronize(run->stream));
    return CHHS_OK;
  }

  // Face velocities into out[0..DIM) (device arrays of ncell values).
  static chhs_status velocity(chhs_t* run, double* const* out) {
    k_velocity<DIM><<<nblocks(run->ncell()), kBlock, 0, run->stream>>>(run->lev[0], run->gamma, 1.0 / run->h,
                                                                         out[0], out[1], out[2]);
    CU(cudaGetLastError());
    return CHHS_OK;
  }

  static chhs_status energy(chhs_t* run) {
    const int nx = run->n[0], ny = run->n[1], nz = run->n[2];
    const int nb = nblocks(run->ncell());
    k_energy_partial<DIM><<<nb, kBlock, 0, run->stream>>>(run->lev[0].phim, run->phimm1, nx, ny, nz,
                                                          1.0 / run->h, run->partials);
    k_energy_finish<<<1, 1024, 0, run->stream>>>(run->partials, nb, run->st);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(run->host_st, run->st, sizeof(DevState), cudaMemcpyDeviceToHost, run->stream));
    CU(cudaStreamSynchronize(run->stream));
    return CHHS_OK;
  }
};

__global__ void k_reset_call(DevState* st, double tol, double tol_max, int max_v, int max_inner) {
  st->failed = 0;
  st->vtotal = 0;
  st->steps_done = 0;
  st->checks = 0;
  st->tol = tol;
  st->tol_max = tol_max;
  st->max_v = max_v;
  st->max_inner = max_inner;
}

// The pointwise guard's bound (infinite when the guard is off).
double tol_max_of(const chhs_opts& o) {
  return o.max_factor > 0 ? o.max_factor * o.tol : INFINITY;
}

// The arrays of one level, carved out of the arena at base.
template <typename T>
Level<T> make_level(const chhs_t* run, const Shape& sh, int l, char* base, bool single) {
  size_t nc = (size_t)sh.n[0] * sh.n[1] * sh.n[2];
  size_t stride = align_up(sizeof(T) * nc);
  const int nf = level_fields(run->dim, single);
  T* f[kBaseFields + 21];
  for (int q = 0; q < nf; ++q) f[q] = reinterpret_cast<T*>(base + q * stride);
  const double hl = run->h * double(1 << l);
  Level<T> L;
  L.phi = f[0]; L.mu = f[1]; L.p = f[2];
  L.fphi = f[3]; L.fmu = f[4]; L.fp = f[5];
  L.phim = f[6]; L.phis = f[7];
  L.phi0 = f[8]; L.mu0 = f[9]; L.p0 = f[10];
  L.ax = f[11]; L.ay = f[12]; L.Mx = f[13]; L.My = f[14];
  L.sM = f[15]; L.sa = f[16];
  L.cAe = f[17]; L.cC = f[18]; L.cGn = f[19]; L.cHn = f[20]; L.cQ = f[21]; L.cH = f[22];
  int q = 23;
  L.az = run->dim == 3 ? f[q++] : nullptr;
  L.Mz = run->dim == 3 ? f[q++] : nullptr;
  L.phib = single ? f[q++] : nullptr;
  const bool tiles = single && run->dim == 2;
  L.phi2 = tiles ? f[q++] : nullptr;
  L.mu2 = tiles ? f[q++] : nullptr;
  L.p2 = tiles ? f[q++] : nullptr;
  L.fc1 = tiles ? f[q++] : nullptr;
  L.fc2 = tiles ? f[q++] : nullptr;
  L.fc3 = tiles ? f[q++] : nullptr;
  L.nx = sh.n[0]; L.ny = sh.n[1]; L.nz = sh.n[2];
  L.ncell = (int)nc;
  L.rnx = 1.0f / (float)sh.n[0];
  L.rny = 1.0f / (float)sh.n[1];
  L.rhw = 1.0f / (float)((sh.n[0] + 1) / 2);
  L.ih2 = T(1.0 / (hl * hl));
  L.h2 = T(hl * hl);
  L.sih2 = T(run->dt / (hl * hl));
  L.e34ih2 = T(0.75 * run->eps * run->eps / (hl * hl));
  return L;
}

template <typename T>
void fill_tail(Tail<T>& tail, const std::vector<Level<T>>& lev, int start, const chhs_opts& o, int nu1c, int nu2c) {
  tail.n = 0;
  for (int l = start; l < (int)lev.size(); ++l) tail.lev[tail.n++] = lev[l];
  tail.nu1 = start > 0 ? nu1c : o.nu1;
  tail.nu2 = start > 0 ? nu2c : o.nu2;
  tail.top_rhs = start > 0 ? 1 : 0;
  tail.coarsest_f64 = (sizeof(T) == 4 && o.coarsest_f64) ? 1 : 0;
}

// The first level of the one-block tail: the coarsest, and every level above
// it with at most tail_cells cells (up to kTailMaxLevels levels).
void place_tail(chhs_t* run) {
  const Layout& Lo = run->layout;
  const int nl = (int)Lo.shapes.size();
  auto cells = [&](int l) { return Lo.shapes[l].n[0] * Lo.shapes[l].n[1] * Lo.shapes[l].n[2]; };
  run->tail_start = nl - 1;
  while (run->tail_start > 0 && cells(run->tail_start - 1) <= run->tail_cells &&
         nl - (run->tail_start - 1) <= kTailMaxLevels)
    --run->tail_start;
  fill_tail(run->tail, run->lev, run->tail_start, run->opts, run->nu1c, run->nu2c);
  fill_tail(run->tail32, run->lev32, run->tail_start, run->opts, run->nu1c, run->nu2c);
}

chhs_status setup_handle(chhs_t* run) {
  const Layout& Lo = run->layout;
  run->st = reinterpret_cast<DevState*>(run->arena + Lo.state_off);
  run->partials = reinterpret_cast<double*>(run->arena + Lo.partial_off);
  run->phimm1 = reinterpret_cast<double*>(run->arena + Lo.phimm1_off);
  for (int l = 0; l < Lo.nlev64; ++l)
    run->lev.push_back(make_level<double>(run, Lo.shapes[l], l, run->arena + Lo.level_off[l], false));
  for (size_t l = 0; l < Lo.level32_off.size(); ++l)
    run->lev32.push_back(make_level<float>(run, Lo.shapes[l], (int)l, run->arena + Lo.level32_off[l], true));
  run->tail_cells = run->opts.precision == 1 ? kTailCellsF32 : kTailCellsF64;
  run->nu1c = run->opts.nu1;
  run->nu2c = run->opts.nu2;
  place_tail(run);
  // The norm kernels loop over cells with the grid's stride: kNormBlocksPerSM
  // blocks on every SM (all resident at once), so no SM holds a block more
  // than another; small grids take one cell per thread.
  int dev = 0, nsm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  run->norm_blocks = std::max(1, std::min(nblocks(run->ncell()), kNormBlocksPerSM * nsm));
  CU(cudaMemsetAsync(run->arena, 0, Lo.total, run->stream));
  CU(cudaMallocHost(&run->host_st, sizeof(DevState)));
  memset(run->host_st, 0, sizeof(DevState));
  if (run->batch_member) return CHHS_OK;  // the batch builds the one graph of all its runs
  chhs_status s = run->dim == 2 ? Enqueue<2>::build_graph(run) : Enqueue<3>::build_graph(run);
  if (s != CHHS_OK) return s;
  CU(cudaStreamSynchronize(run->stream));
  return CHHS_OK;
}

chhs_status create_impl(int dim, const int n[3], double h, double eps, double gamma, double dt,
                        const chhs_opts* opts, void* cuda_stream, void* arena, size_t arena_bytes,
                        chhs_t** out, bool member = false) {
  if (!out) return CHHS_ERR_INVALID_ARG;
  *out = nullptr;
  chhs_opts o;
  chhs_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_problem(dim, n, h, eps, gamma, dt) || !valid_opts(o)) return CHHS_ERR_INVALID_ARG;
  const int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  Layout layout = make_layout(dim, nn, o.coarsest, o.precision);
  if (arena) {  // the caller's arena is checked before any CUDA call
    if (reinterpret_cast<uintptr_t>(arena) % kAlign != 0) return CHHS_ERR_INVALID_ARG;
    if (arena_bytes < layout.total) return CHHS_ERR_OOM;
  }
  chhs_t* run = new (std::nothrow) chhs_t();
  if (!run) return CHHS_ERR_OOM;
  run->dim = dim;
  for (int a = 0; a < 3; ++a) run->n[a] = nn[a];
  run->h = h; run->eps = eps; run->gamma = gamma; run->dt = dt;
  run->opts = o;
  run->layout = std::move(layout);
  run->batch_member = member;
  chhs_status s = CHHS_OK;
  if (cuda_stream) {
    run->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&run->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete run;
      return CHHS_ERR_CUDA;
    }
    run->own_stream = true;
  }
  if (arena) {
    run->arena = static_cast<char*>(arena);
  } else {
    if (cudaMalloc(&run->arena, run->layout.total) != cudaSuccess) {
      cudaGetLastError();
      run->arena = nullptr;
      destroy_handle(run);
      return CHHS_ERR_OOM;
    }
    run->own_arena = true;
  }
  s = setup_handle(run);
  if (s != CHHS_OK) {
    destroy_handle(run);
    return s;
  }
  *out = run;
  return CHHS_OK;
}

// A handle's launch settings as a chhs_tuning, and back (ms_per_step unused).
chhs_tuning current_tuning(const chhs_t* run) {
  chhs_tuning t{};
  t.tail_cells = run->tail_cells;
  t.split_threads = run->split_threads;
  t.tile_threads = run->tile_threads;
  t.coarse_nu1 = run->nu1c;
  t.coarse_nu2 = run->nu2c;
  t.tile_w = run->tile_w;
  t.tile_h = run->tile_h;
  t.norm_f64_per8 = run->norm_f64_per8;
  t.small_tile_w = run->stile_w;
  t.small_tile_h = run->stile_h;
  t.small_tile_threads = run->stile_threads;
  t.quad_passes = run->quad_passes;
  t.ms_per_step = -1.0;
  return t;
}

void take_tuning(chhs_t* run, const chhs_tuning& t) {
  run->tail_cells = t.tail_cells;
  run->split_threads = t.split_threads;
  run->tile_threads = t.tile_threads;
  run->nu1c = t.coarse_nu1;
  run->nu2c = t.coarse_nu2;
  run->tile_w = t.tile_w;
  run->tile_h = t.tile_h;
  run->norm_f64_per8 = t.norm_f64_per8;
  run->stile_w = t.small_tile_w;
  run->stile_h = t.small_tile_h;
  run->stile_threads = t.small_tile_threads;
  run->quad_passes = t.quad_passes;
}

chhs_status copy_in(chhs_t* run, double* dst, const double* src, int on_device) {
  size_t bytes = sizeof(double) * run->ncell();
  CU(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     run->stream));
  return CHHS_OK;
}

chhs_status copy_out(chhs_t* run, double* dst, const double* src, int on_device) {
  size_t bytes = sizeof(double) * run->ncell();
  CU(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     run->stream));
  return CHHS_OK;
}

}  // namespace

extern "C" {

chhs_status chhs_default_opts(chhs_opts* o) {
  if (!o) return CHHS_ERR_INVALID_ARG;
  o->nu1 = 2;
  o->nu2 = 2;
  o->max_v = 50;
  o->coarsest = 2;
  o->tol = 1e-10;
  o->precision = 0;
  o->max_factor = 50.0;
  o->coarsest_f64 = 0;
  o->f64_residual = 0;
  o->max_inner = 3;  // kMaxInner (4) measured no faster on the benchmark workloads
  return CHHS_OK;
}

size_t chhs_workspace_bytes(int dim, const int n[3], const chhs_opts* opts) {
  chhs_opts o;
  chhs_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_problem(dim, n, 1.0, 1.0, 0.0, 1.0) || !valid_opts(o)) return 0;
  int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  return make_layout(dim, nn, o.coarsest, o.precision).total;
}

chhs_status chhs_create(int dim, const int n[3], double h, double eps, double gamma, double dt,
                        const chhs_opts* opts, void* cuda_stream, chhs_t** out) {
  return create_impl(dim, n, h, eps, gamma, dt, opts, cuda_stream, nullptr, 0, out);
}

chhs_status chhs_create_ext(int dim, const int n[3], double h, double eps, double gamma, double dt,
                            const chhs_opts* opts, void* cuda_stream, void* arena, size_t arena_bytes,
                            chhs_t** out) {
  if (!arena) return CHHS_ERR_INVALID_ARG;
  return create_impl(dim, n, h, eps, gamma, dt, opts, cuda_stream, arena, arena_bytes, out);
}

chhs_status chhs_set_phi(chhs_t* run, const double* phi0, const double* phi_prev, int on_device) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  if (!phi0) return fail(run, CHHS_ERR_INVALID_ARG, "phi0 is NULL");
  return chhs_set_state(run, phi0, phi_prev ? phi_prev : phi0, nullptr, nullptr, on_device);
}

chhs_status chhs_set_state(chhs_t* run, const double* phi, const double* phi_prev, const double* mu,
                           const double* p, int on_device) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  if (!phi || !phi_prev) return fail(run, CHHS_ERR_INVALID_ARG, "phi and phi_prev are required");
  run->err.clear();
  const Level<double>& F = run->lev[0];
  size_t bytes = sizeof(double) * run->ncell();
  chhs_status s;
  if ((s = copy_in(run, F.phim, phi, on_device)) != CHHS_OK) return s;
  if ((s = copy_in(run, run->phimm1, phi_prev, on_device)) != CHHS_OK) return s;
  if (mu) {
    if ((s = copy_in(run, F.mu, mu, on_device)) != CHHS_OK) return s;
  } else {
    CU(cudaMemsetAsync(F.mu, 0, bytes, run->stream));
  }
  if (p) {
    if ((s = copy_in(run, F.p, p, on_device)) != CHHS_OK) return s;
  } else {
    CU(cudaMemsetAsync(F.p, 0, bytes, run->stream));
  }
  if (!on_device) CU(cudaStreamSynchronize(run->stream));
  return CHHS_OK;
}

chhs_status chhs_step_async(chhs_t* run, int nsteps) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  if (run->batch_member) return fail(run, CHHS_ERR_INVALID_ARG, "a run of a batch is stepped by chhs_batch_step");
  if (nsteps < 0) return fail(run, CHHS_ERR_INVALID_ARG, "nsteps < 0");
  run->err.clear();
  if (!run->pending) {  // the first call since the last wait starts a new count
    k_reset_call<<<1, 1, 0, run->stream>>>(run->st, run->opts.tol, tol_max_of(run->opts), run->opts.max_v,
                                           run->opts.max_inner);
    CU(cudaGetLastError());
    run->pending = true;
  }
  for (int k = 0; k < nsteps; ++k) CU(cudaGraphLaunch(run->exec, run->stream));
  return CHHS_OK;
}

chhs_status chhs_wait(chhs_t* run, int* vcycles_out, double* resid_out) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  run->pending = false;
  CU(cudaMemcpyAsync(run->host_st, run->st, sizeof(DevState), cudaMemcpyDeviceToHost, run->stream));
  CU(cudaStreamSynchronize(run->stream));
  const DevState& h = *run->host_st;
  if (vcycles_out) *vcycles_out = h.vtotal + (h.failed ? h.vcycles : 0);
  if (resid_out) *resid_out = h.resid;
  if (h.failed == CHHS_ERR_NOT_CONVERGED) {
    char b[160];
    snprintf(b, sizeof b, "step %d: residual %.3e above tol %.3e after %d V-cycles", h.steps_done + 1,
             h.resid, run->opts.tol, h.vcycles);
    return fail(run, CHHS_ERR_NOT_CONVERGED, b);
  }
  if (h.failed == CHHS_ERR_DIVERGED) {
    char b[160];
    snprintf(b, sizeof b, "step %d: residual diverged (%.3e)", h.steps_done + 1, h.resid);
    return fail(run, CHHS_ERR_DIVERGED, b);
  }
  return CHHS_OK;
}

chhs_status chhs_step(chhs_t* run, int nsteps, int* vcycles_out, double* resid_out) {
  chhs_status s = chhs_step_async(run, nsteps);
  if (s != CHHS_OK) return s;
  return chhs_wait(run, vcycles_out, resid_out);
}

chhs_status chhs_launch_counts(const chhs_t* run, int* per_vcycle, int* per_step) {
  if (!run || !per_vcycle || !per_step) return CHHS_ERR_INVALID_ARG;
  *per_vcycle = run->launches_per_v;
  *per_step = run->launches_per_step;
  return CHHS_OK;
}

chhs_status chhs_norm_checks(const chhs_t* run, int* checks) {
  if (!run || !checks) return CHHS_ERR_INVALID_ARG;
  *checks = run->host_st ? run->host_st->checks : 0;
  return CHHS_OK;
}

chhs_status chhs_profile_step(chhs_t* run, double* ms_out, long long* launches_out, double* units_out) {
  if (!run || !ms_out || !launches_out || !units_out) return fail(run, CHHS_ERR_INVALID_ARG, "NULL argument");
  // it resets the step counters, which would drop a pending step's status
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  run->err.clear();
  Prof prof;
  run->prof = &prof;
  k_reset_call<<<1, 1, 0, run->stream>>>(run->st, run->opts.tol, tol_max_of(run->opts), run->opts.max_v,
                                         run->opts.max_inner);
  chhs_status s = run->dim == 2 ? Enqueue<2>::profile_step(run) : Enqueue<3>::profile_step(run);
  run->prof = nullptr;
  if (s != CHHS_OK) return s;
  for (size_t q = 0; q < prof.kind.size(); ++q) {
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, prof.ev[2 * q], prof.ev[2 * q + 1]));
    ms_out[prof.kind[q]] += ms;
    launches_out[prof.kind[q]] += 1;
    units_out[prof.kind[q]] += prof.units[q];
  }
  return chhs_wait(run, nullptr, nullptr);
}

chhs_status chhs_profile_smooth(chhs_t* run, int npasses, double* ms_per_pass) {
  if (!run || npasses < 1 || !ms_per_pass) return fail(run, CHHS_ERR_INVALID_ARG, "bad argument");
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  run->err.clear();
  struct Events {  // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CU(cudaEventCreate(&ev.a));
  CU(cudaEventCreate(&ev.b));
  const Level<double>& L = run->lev[0];
  const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
  const int blocks = (threads + kSmoothBlock - 1) / kSmoothBlock;
  const Coefs<double> K{run->dt, run->gamma, 0.75 * run->eps * run->eps};
  // the passes overwrite (phi, mu, p) of the finest level: keep a copy in the
  // finest level's R u arrays (only the coarse levels use theirs) and put it back
  const size_t bytes = sizeof(double) * (size_t)L.ncell;
  CU(cudaMemcpyAsync(L.phi0, L.phi, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.mu0, L.mu, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.p0, L.p, bytes, cudaMemcpyDeviceToDevice, run->stream));
  // one untimed pass, then npasses timed ones back to back
  for (int k = 0; k <= npasses; ++k) {
    if (k == 1) CU(cudaEventRecord(ev.a, run->stream));
    if (run->dim == 2)
      pdl(k_smooth<double, 2, false>, blocks, kSmoothBlock, run->stream, L, K, k & 1, 0);
    else
      pdl(k_smooth<double, 3, false>, blocks, kSmoothBlock, run->stream, L, K, k & 1, 0);
  }
  CU(cudaGetLastError());
  CU(cudaEventRecord(ev.b, run->stream));
  CU(cudaMemcpyAsync(L.phi, L.phi0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.mu, L.mu0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.p, L.p0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaStreamSynchronize(run->stream));
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, ev.a, ev.b));
  *ms_per_pass = ms / npasses;
  return CHHS_OK;
}

chhs_status chhs_profile_smooth32(chhs_t* run, int npasses, double* ms_per_launch) {
  if (!run || npasses < 1 || !ms_per_launch) return fail(run, CHHS_ERR_INVALID_ARG, "bad argument");
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  if (run->opts.precision != 1 || run->tail_start == 0)
    return fail(run, CHHS_ERR_INVALID_ARG, "needs a mixed-precision handle whose finest level is not in the tail");
  run->err.clear();
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CU(cudaEventCreate(&ev.a));
  CU(cudaEventCreate(&ev.b));
  const Level<float>& L = run->lev32[0];
  const Level<float>& C = run->lev32[1];
  const Coefs<float> K{(float)run->dt, (float)run->gamma, (float)(0.75 * run->eps * run->eps)};
  // the finest single-precision level's correction is scratch between steps
  // (the stopping norm rewrites it), but it is kept and put back all the same
  // (in its R u arrays, which only the coarser levels use); the launches also
  // write the next level and the tiles' second copy, which every V-cycle
  // rewrites before reading
  const size_t bytes = sizeof(float) * (size_t)L.ncell;
  CU(cudaMemcpyAsync(L.phi0, L.phi, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.mu0, L.mu, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.p0, L.p, bytes, cudaMemcpyDeviceToDevice, run->stream));
  const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
  const int blocks = (threads + kSmoothBlock - 1) / kSmoothBlock;
  const int np1 = 2 * run->opts.nu1;
  const TileOut<float> to_copy{L.phi2, L.mu2, L.p2, L.fc1, L.fc2, L.fc3, nullptr, nullptr, nullptr};
  const bool large = L.ncell >= kLargeTileCells;
  const int tw = large ? run->tile_w : run->stile_w, th = large ? run->tile_h : run->stile_h;
  const int tt = large ? run->tile_threads : run->stile_threads;
  const dim3 grid((L.nx + tw - 1) / tw, (L.ny + th - 1) / th);
  for (int k = 0; k <= npasses; ++k) {
    if (k == 1) CU(cudaEventRecord(ev.a, run->stream));
    if (run->dim == 3 && Enqueue<3>::quad_level(run, L))
      pdl_grid(k_smooth_c4<0, 0>, quad_grid(L.nx, L.ny, L.nz), kSmoothBlock, 0, run->stream, L, C, K, k & 1,
               Level<double>{}, quad_tile(L.nx));
    else if (run->dim == 3)
      pdl(k_smooth_c<3>, blocks, kSmoothBlock, run->stream, L, C, K, k & 1, 0, 0, Level<double>{});
    else
      pdl_grid(k_tile<float, true>, grid, tt, tile_smem_bytes(np1 + 1, tile_nfields<true>(), 4, tw, th),
               run->stream, L, C, K, np1, np1 + 1, 0, 0, 1, to_copy, (const int*)nullptr, tw, th);
  }
  CU(cudaGetLastError());
  CU(cudaEventRecord(ev.b, run->stream));
  CU(cudaMemcpyAsync(L.phi, L.phi0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.mu, L.mu0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaMemcpyAsync(L.p, L.p0, bytes, cudaMemcpyDeviceToDevice, run->stream));
  CU(cudaStreamSynchronize(run->stream));
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, ev.a, ev.b));
  *ms_per_launch = ms / npasses;
  return CHHS_OK;
}

// Throughput of the FP64 pipe: every thread runs 8 independent chains of
// fused multiply-adds (x <- x a + b) in double precision.
__global__ void k_fp64_probe(double a, double b, int iters, double* sink) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == 12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
}

chhs_status chhs_probe_fp64(double* tflops_out) {
  chhs_t* run = nullptr;
  if (!tflops_out) return CHHS_ERR_INVALID_ARG;
  int dev = 0, nsm = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  k_fp64_probe<<<blocks, threads>>>(0.999999, 1e-7, 64, nullptr);  // warm-up
  cudaEventRecord(e0);
  k_fp64_probe<<<blocks, threads>>>(0.999999, 1e-7, iters, nullptr);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return CHHS_ERR_CUDA;
  *tflops_out = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return CHHS_OK;
}

// Read bandwidth of the L2: every thread sums 16-byte words of a buffer that
// fits in the L2, bypassing L1 (ld.global.cg), for `passes` passes.
__global__ void k_l2_probe(const float4* buf, long long n4, int passes, float* sink) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  float acc = 0.f;
  for (int p = 0; p < passes; ++p)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  if (acc == 12345.678f) sink[0] = acc;  // keeps the loads live; the buffer holds zeros
}

chhs_status chhs_probe_l2(size_t bytes, int passes, double* gbs_out) {
  chhs_t* run = nullptr;  // no handle: CU reports the status only
  if (!gbs_out || passes < 1 || bytes < (1u << 20) || bytes > ((size_t)1 << 30)) return CHHS_ERR_INVALID_ARG;
  int dev = 0, nsm = 0, l2 = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CU(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  if (bytes > (size_t)l2 / 2) return CHHS_ERR_INVALID_ARG;
  struct Res {
    float4* buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    ~Res() {
      if (buf) cudaFree(buf);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } r;
  const long long n4 = (long long)(bytes / sizeof(float4));
  if (cudaMalloc(&r.buf, (size_t)n4 * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    return CHHS_ERR_OOM;
  }
  CU(cudaMemset(r.buf, 0, (size_t)n4 * sizeof(float4)));
  CU(cudaEventCreate(&r.a));
  CU(cudaEventCreate(&r.b));
  const int blocks = nsm * 8, threads = 256;
  k_l2_probe<<<blocks, threads>>>(r.buf, n4, 2, nullptr);  // brings the buffer into the L2
  CU(cudaEventRecord(r.a));
  k_l2_probe<<<blocks, threads>>>(r.buf, n4, passes, nullptr);
  CU(cudaEventRecord(r.b));
  CU(cudaEventSynchronize(r.b));
  CU(cudaGetLastError());
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, r.a, r.b));
  *gbs_out = (double)n4 * sizeof(float4) * passes / (ms * 1e-3) / 1e9;
  return CHHS_OK;
}

chhs_status chhs_set_tuning(chhs_t* run, const chhs_tuning* t) {
  if (!run || !t) return fail(run, CHHS_ERR_INVALID_ARG, "NULL argument");
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  if (run->batch_member) return fail(run, CHHS_ERR_INVALID_ARG, "a run of a batch takes the batch's launch shapes");
  auto tile_ok = [](int w, int h, int threads) {
    return threads >= 32 && threads <= 1024 && threads % 32 == 0 && w >= 2 && h >= 2 && w % 2 == 0 && h % 2 == 0 &&
           w * h <= 4096;
  };
  if (t->tail_cells < 1 || t->split_threads < 0 || t->coarse_nu1 < 0 || t->coarse_nu2 < 0 ||
      t->coarse_nu1 + t->coarse_nu2 < 1 || !tile_ok(t->tile_w, t->tile_h, t->tile_threads) ||
      !tile_ok(t->small_tile_w, t->small_tile_h, t->small_tile_threads) || t->norm_f64_per8 < 0 ||
      t->norm_f64_per8 > 8 || (t->quad_passes != 0 && t->quad_passes != 1))
    return fail(run, CHHS_ERR_INVALID_ARG, "invalid tuning");
  run->norm_f64_per8 = t->norm_f64_per8;
  run->err.clear();
  CU(cudaStreamSynchronize(run->stream));
  const chhs_tuning keep = current_tuning(run);
  auto rebuild = [&](const chhs_tuning& c) -> chhs_status {
    if (run->exec) cudaGraphExecDestroy(run->exec);
    if (run->graph) cudaGraphDestroy(run->graph);
    run->exec = nullptr;
    run->graph = nullptr;
    take_tuning(run, c);
    place_tail(run);
    return run->dim == 2 ? Enqueue<2>::build_graph(run) : Enqueue<3>::build_graph(run);
  };
  chhs_status s = rebuild(*t);
  if (s != CHHS_OK) {
    const std::string why = run->err;
    if (rebuild(keep) != CHHS_OK) return fail(run, CHHS_ERR_CUDA, "could not rebuild the step graph");
    return fail(run, s, why.empty() ? "tuning refused" : why);
  }
  return CHHS_OK;
}

chhs_status chhs_autotune(chhs_t* run, int trial_steps, chhs_tuning* out) {
  if (!run || trial_steps < 1) return fail(run, CHHS_ERR_INVALID_ARG, "bad argument");
  if (run->batch_member) return fail(run, CHHS_ERR_INVALID_ARG, "a run of a batch takes the batch's launch shapes");
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  run->err.clear();
  using Cand = chhs_tuning;
  std::vector<Cand> cands;
  const chhs_tuning base = current_tuning(run);
  auto cand = [&](int tc, int sp, int tt, int n1, int n2, int tw, int th, int ctw, int cth, int ctt) {
    chhs_tuning c = base;
    c.tail_cells = tc;
    c.split_threads = sp;
    c.tile_threads = tt;
    c.coarse_nu1 = n1;
    c.coarse_nu2 = n2;
    c.tile_w = tw;
    c.tile_h = th;
    c.small_tile_w = ctw;
    c.small_tile_h = cth;
    c.small_tile_threads = ctt;
    cands.push_back(c);
  };
  const bool mixed = run->opts.precision == 1;
  // sweep counts below the finest level: the options' own, and one sweep
  // each way when the options ask for more (fewer passes on the small,
  // latency-bound levels; the V-cycle counts the trials measure decide)
  std::vector<std::pair<int, int>> coarse = {{run->opts.nu1, run->opts.nu2}};
  if (run->opts.nu1 > 1 && run->opts.nu2 > 1) coarse.push_back({1, 1});
  // 2D mixed form: tile shapes (interior cells; wider tiles recompute a
  // smaller share of halo cells but make fewer blocks) and block sizes
  struct Shape2 {
    int tt, tw, th;
  };
  const Shape2 shapes[4] = {{256, 32, 16}, {512, 32, 16}, {512, 32, 32}, {512, 64, 16}};
  // the levels under kLargeTileCells: the same shape, or the small one
  const Shape2 small{kSmallTileThreads, kSmallTileW, kSmallTileH};
  for (const auto& cn : coarse) {
    if (!mixed) {
      const int tails[2] = {64, run->dim == 2 ? 256 : 512};
      for (int tc : tails)
        for (int sp : {0, 8192, 32768})
          cand(tc, sp, run->tile_threads, cn.first, cn.second, run->tile_w, run->tile_h, run->stile_w, run->stile_h,
               run->stile_threads);
    } else if (run->dim == 2) {
      for (int tc : {256, 1024, 2048})
        for (const Shape2& sh : shapes)
          for (const Shape2& cs : {sh, small})
            cand(tc, run->split_threads, sh.tt, cn.first, cn.second, sh.tw, sh.th, cs.tw, cs.th, cs.tt);
    } else {
      for (int tc : {64, 512})
        cand(tc, run->split_threads, run->tile_threads, cn.first, cn.second, run->tile_w, run->tile_h, run->stile_w,
             run->stile_h, run->stile_threads);
    }
  }
  // the run's state (phi^m, phi^{m-1}, mu, p), restored before every trial and at the end
  const size_t nc = (size_t)run->ncell(), bytes = sizeof(double) * nc;
  double* keep = nullptr;
  if (cudaMalloc(&keep, 4 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(run, CHHS_ERR_OOM, "no room for the state copy");
  }
  struct Free {
    double* p;
    ~Free() { cudaFree(p); }
  } free_keep{keep};
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CU(cudaEventCreate(&ev.a));
  CU(cudaEventCreate(&ev.b));
  const Level<double>& F = run->lev[0];
  double* state[4] = {F.phim, run->phimm1, F.mu, F.p};
  for (int q = 0; q < 4; ++q)
    CU(cudaMemcpyAsync(keep + q * nc, state[q], bytes, cudaMemcpyDeviceToDevice, run->stream));
  auto restore = [&]() -> chhs_status {
    for (int q = 0; q < 4; ++q)
      CU(cudaMemcpyAsync(state[q], keep + q * nc, bytes, cudaMemcpyDeviceToDevice, run->stream));
    return CHHS_OK;
  };
  auto apply = [&](const Cand& c) -> chhs_status {
    CU(cudaStreamSynchronize(run->stream));
    if (run->exec) cudaGraphExecDestroy(run->exec);
    if (run->graph) cudaGraphDestroy(run->graph);
    run->exec = nullptr;
    run->graph = nullptr;
    take_tuning(run, c);
    place_tail(run);
    return run->dim == 2 ? Enqueue<2>::build_graph(run) : Enqueue<3>::build_graph(run);
  };
  const Cand orig = base;
  Cand best = orig;
  float best_ms = -1.f;
  chhs_status s;
  for (const Cand& c : cands) {
    if (apply(c) != CHHS_OK) continue;  // e.g. a tail too large for shared memory
    if ((s = restore()) != CHHS_OK) return s;
    if (chhs_step(run, 1, nullptr, nullptr) != CHHS_OK) continue;  // warm-up
    if ((s = restore()) != CHHS_OK) return s;
    CU(cudaEventRecord(ev.a, run->stream));
    const chhs_status sa = chhs_step_async(run, trial_steps);
    CU(cudaEventRecord(ev.b, run->stream));
    if (chhs_wait(run, nullptr, nullptr) != CHHS_OK || sa != CHHS_OK) continue;
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, ev.a, ev.b));
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  run->err.clear();
  if ((s = apply(best)) != CHHS_OK) {
    // the fastest setting could not be rebuilt: the original one is kept, and
    // its time is not the one measured for the best candidate
    if (apply(orig) != CHHS_OK) return fail(run, CHHS_ERR_CUDA, "could not rebuild the step graph");
    best_ms = -1.f;
  }
  if ((s = restore()) != CHHS_OK) return s;
  CU(cudaStreamSynchronize(run->stream));
  if (out) {
    *out = current_tuning(run);
    out->ms_per_step = best_ms < 0.f ? -1.0 : (double)best_ms / trial_steps;
  }
  return CHHS_OK;
}

chhs_status chhs_mass(chhs_t* run, double* mass_out) {
  if (!run || !mass_out) return fail(run, CHHS_ERR_INVALID_ARG, "NULL argument");
  run->err.clear();
  chhs_status s = run->dim == 2 ? Enqueue<2>::energy(run) : Enqueue<3>::energy(run);
  if (s != CHHS_OK) return s;
  double hd = run->dim == 2 ? run->h * run->h : run->h * run->h * run->h;
  *mass_out = hd * run->host_st->diag[0];
  return CHHS_OK;
}

chhs_status chhs_energy(chhs_t* run, double* E_out, double* F_out) {
  if (!run || !E_out) return fail(run, CHHS_ERR_INVALID_ARG, "NULL argument");
  run->err.clear();
  chhs_status s = run->dim == 2 ? Enqueue<2>::energy(run) : Enqueue<3>::energy(run);
  if (s != CHHS_OK) return s;
  const double* d = run->host_st->diag;
  double hd = run->dim == 2 ? run->h * run->h : run->h * run->h * run->h;
  double e2 = run->eps * run->eps;
  // Eq. 2.8: E_h = 1/4 ||phi||_4^4 - 1/2 ||phi||_2^2 + eps^2/2 ||grad_h phi||_2^2
  double E = 0.25 * hd * d[1] - 0.5 * hd * d[2] + 0.5 * e2 * hd * d[3];
  *E_out = E;
  // Eq. 2.9: F_h = E_h + 1/4 ||phi - psi||^2 + 1/8 eps^2 ||grad_h(phi - psi)||^2
  if (F_out) *F_out = E + 0.25 * hd * d[4] + 0.125 * e2 * hd * d[5];
  return CHHS_OK;
}

chhs_status chhs_dissipation(chhs_t* run, double* grad_mu_sq, double* u_sq, double* div_u_max) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  run->err.clear();
  chhs_status s = run->dim == 2 ? Enqueue<2>::dissipation(run) : Enqueue<3>::dissipation(run);
  if (s != CHHS_OK) return s;
  const double* d = run->host_st->diag;
  double hd = run->dim == 2 ? run->h * run->h : run->h * run->h * run->h;
  if (grad_mu_sq) *grad_mu_sq = hd * d[0];
  if (u_sq) *u_sq = hd * d[1];
  if (div_u_max) *div_u_max = d[2];
  return CHHS_OK;
}

chhs_status chhs_velocity(chhs_t* run, double* ux, double* uy, double* uz, int on_device) {
  if (!run || !ux || !uy || (run->dim == 3 && !uz)) return fail(run, CHHS_ERR_INVALID_ARG, "bad argument");
  if (run->pending) return fail(run, CHHS_ERR_INVALID_ARG, "steps pending: call chhs_wait first");
  run->err.clear();
  double* dst[3] = {ux, uy, run->dim == 3 ? uz : nullptr};
  // host outputs are staged in the finest level's R u arrays, which only the
  // coarse levels use
  const Level<double>& F = run->lev[0];
  double* stage[3] = {F.phi0, F.mu0, F.p0};
  double* out[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < run->dim; ++a) out[a] = on_device ? dst[a] : stage[a];
  chhs_status s = run->dim == 2 ? Enqueue<2>::velocity(run, out) : Enqueue<3>::velocity(run, out);
  if (s != CHHS_OK) return s;
  if (!on_device)
    for (int a = 0; a < run->dim; ++a)
      if ((s = copy_out(run, dst[a], stage[a], 0)) != CHHS_OK) return s;
  CU(cudaStreamSynchronize(run->stream));
  return CHHS_OK;
}

chhs_status chhs_get_phi(chhs_t* run, double* out, int on_device) {
  return chhs_get_state(run, out, nullptr, nullptr, nullptr, on_device);
}

chhs_status chhs_get_state(chhs_t* run, double* phi, double* phi_prev, double* mu, double* p,
                           int on_device) {
  if (!run) return CHHS_ERR_INVALID_ARG;
  run->err.clear();
  const Level<double>& F = run->lev[0];
  chhs_status s;
  if (phi && (s = copy_out(run, phi, F.phim, on_device)) != CHHS_OK) return s;
  if (phi_prev && (s = copy_out(run, phi_prev, run->phimm1, on_device)) != CHHS_OK) return s;
  if (mu && (s = copy_out(run, mu, F.mu, on_device)) != CHHS_OK) return s;
  if (p && (s = copy_out(run, p, F.p, on_device)) != CHHS_OK) return s;
  if (!on_device) CU(cudaStreamSynchronize(run->stream));
  return CHHS_OK;
}

int chhs_num_levels(const chhs_t* run) { return run ? (int)run->lev.size() : 0; }

void chhs_destroy(chhs_t* run) {
  if (!run || run->batch_member) return;  // a batch's runs are released with the batch
  destroy_handle(run);
}

}  // extern "C"

namespace {

void destroy_handle(chhs_t* run) {
  if (run->stream) cudaStreamSynchronize(run->stream);
  if (run->exec) cudaGraphExecDestroy(run->exec);
  if (run->graph) cudaGraphDestroy(run->graph);
  if (run->host_st) cudaFreeHost(run->host_st);
  if (run->own_arena && run->arena) cudaFree(run->arena);
  if (run->own_stream && run->stream) cudaStreamDestroy(run->stream);
  delete run;
}

}  // namespace

extern "C" const char* chhs_last_error(const chhs_t* run) { return run ? run->err.c_str() : "NULL handle"; }

// ------------------------------------------------------------------ batches
//
// chhs_batch_*: many independent runs of the mixed-precision form stepped by
// one CUDA graph.  Each launch of the graph covers one kernel of one
// multigrid level for every run that has that level (chhs_batch.cuh): level
// l of the V-cycle is one launch over all runs' level l, all runs' coarse
// tails are one launch of one block per run, and the stopping norms of all
// runs are one launch whose last block keeps the loop going while any run is
// still iterating.  Runs that have converged drop out of the launches (their
// blocks return at once), so each run takes exactly the V-cycles it takes
// alone, and the per-run work is the same device code with the same block
// shapes as its own graph: a run's results are bit-identical to a solo run
// with the same options.

struct chhs_batch {
  int dim = 2, nruns = 0;
  chhs_opts opts{};
  std::vector<chhs_t*> runs;
  char* arena = nullptr;            // every run's hierarchy
  char* tables = nullptr;           // job tables of the batched launches
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevState** d_sts = nullptr;       // per run, for the reset and gather kernels
  unsigned int* d_ticket = nullptr; // blocks of a batched norm launch that have finished
  BatchConds* d_conds = nullptr;    // the step graph's loop and IF conditions
  int* d_out = nullptr;             // status[n], vcycles[n], then resid[n] (doubles)
  char* h_out = nullptr;            // pinned mirror of d_out
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches_per_v = 0, launches_per_step = 0;
  // tile shape of the per-run tile launches of large 2D levels (the batched
  // launch of the small levels keeps 32 x 16 on 512 threads); 32 x 32 took
  // the batched configuration from 6.3e8 to 7.2e8 cell-steps/s
  int big_tw = 32, big_th = 32, big_tt = kTileThreads;
  std::string err;
};

namespace {

chhs_status bfail(chhs_batch_t* b, chhs_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

#define BCU(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bfail(b, CHHS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// Jobs of one batched launch and the prefix sum of their block counts.
template <class J>
struct JobList {
  std::vector<J> jobs;
  std::vector<int> start{0};
  void add(const J& j, int blocks) {
    jobs.push_back(j);
    start.push_back(start.back() + blocks);
  }
  int njobs() const { return (int)jobs.size(); }
  int blocks() const { return start.back(); }
};

// The batch's step, written once and walked twice: first to lay out the job
// tables (plan), then to launch into the capture stream with the tables'
// device addresses (capture), in the same order.
template <int DIM>
struct BatchStep {
  chhs_batch_t* b;
  bool capture = false;
  // the V-cycle being emitted: 1 ends an iteration (gate go, with the
  // update u <- u + e), 2 .. kMaxInner are the extra V-cycles before it
  // (gates go_more[vk - 2], no update) that a run takes when its norm
  // predicted them
  int vk = 1;
  const int* gate(const chhs_t* r) const { return vk == 1 ? &r->st->go : &r->st->go_more[vk - 2]; }
  int n_if() const { return std::min(b->opts.max_inner, kMaxInner) - 1; }
  size_t vstart[kMaxInner + 1] = {};  // table positions of the V-cycles vk = 1..kMaxInner and the norm after them (plan)
  std::vector<char> buf;            // host image of the job tables
  std::vector<size_t> offs;         // table offsets in emission order
  size_t cur = 0;
  int* counter = nullptr;           // launches, while capturing
  size_t tile_smem = 0, tile_smem_big = 0, tail_smem = 0;

  size_t put(const void* p, size_t n) {
    const size_t off = align_up(buf.size());
    buf.resize(off + n);
    if (n) memcpy(buf.data() + off, p, n);
    return off;
  }

  // Launch one batched kernel (or, when planning, lay out its tables).
  template <class J, typename... KArgs, typename... Args>
  void go(int kind, const JobList<J>& jl, void (*kernel)(KArgs...), int block, size_t smem, cudaStream_t s,
          Args... extra) {
    if (jl.jobs.empty()) return;
    if (!capture) {
      offs.push_back(put(jl.jobs.data(), sizeof(J) * jl.jobs.size()));
      offs.push_back(put(jl.start.data(), sizeof(int) * jl.start.size()));
      return;
    }
    const J* dj = reinterpret_cast<const J*>(b->tables + offs[cur++]);
    const int* ds = reinterpret_cast<const int*>(b->tables + offs[cur++]);
    if (counter) ++*counter;
    timed(kind, [&] { pdl_smem(kernel, jl.blocks(), block, smem, s, dj, ds, jl.njobs(), extra...); }, s);
  }

  // Event pairs around the launches while profiling (chhs_batch_profile_step).
  Prof* prof = nullptr;
  template <class F>
  void timed(int kind, F&& f, cudaStream_t s) {
    if (!prof) {
      f();
      return;
    }
    cudaEvent_t a = prof->next(), e = prof->next();
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(e, s);
    prof->kind.push_back(kind);
    prof->units.push_back(1.0);
  }

  // The tail launch: one block per job, no prefix sum.
  void go_tail(const std::vector<TailJob<float>>& jobs, cudaStream_t s) {
    if (jobs.empty()) return;
    if (!capture) {
      offs.push_back(put(jobs.data(), sizeof(TailJob<float>) * jobs.size()));
      return;
    }
    const TailJob<float>* dj = reinterpret_cast<const TailJob<float>*>(b->tables + offs[cur++]);
    if (counter) ++*counter;
    timed(CHHS_K_COARSEST, [&] { pdl_smem(kb_tail<float, DIM, true>, (int)jobs.size(), kTailThreads, tail_smem, s, dj); },
          s);
  }

  static Coefs<float> k32(const chhs_t* r) { return Enqueue<DIM>::template coefs<float>(r); }
  static Coefs<double> k64(const chhs_t* r) { return Enqueue<DIM>::template coefs<double>(r); }

  int max_tail_start() const {
    int m = 0;
    for (const chhs_t* r : b->runs) m = std::max(m, r->tail_start);
    return m;
  }

  void setup(cudaStream_t s) {
    JobList<SetupJob> jl;
    for (chhs_t* r : b->runs) {
      const Level<double>& F = r->lev[0];
      jl.add(SetupJob{F, F, r->phimm1, r->eps * r->eps, r->st, k64(r), 0}, nblocks(F.ncell));
    }
    go(CHHS_K_FRAME, jl, kb_setup_coef<DIM>, kBlock, 0, s);
  }

  void coefs(cudaStream_t s) {
    JobList<CoefF32Job> jf;
    int maxng = 0;
    for (chhs_t* r : b->runs) {
      const int ng = (int)r->lev32.size();
      maxng = std::max(maxng, ng);
      jf.add(CoefF32Job{r->lev[0], r->lev32[0], ng > 1 ? r->lev32[1] : r->lev32[0], k32(r), ng > 1 ? 1 : 0},
             nblocks(r->lev[0].ncell));
    }
    go(CHHS_K_FRAME, jf, kb_coef_restrict_f32<DIM>, kBlock, 0, s);
    for (int l = 1; l < maxng; ++l) {
      JobList<CoefJob> jl;
      for (chhs_t* r : b->runs) {
        const int ng = (int)r->lev32.size();
        if (l >= ng) continue;
        const Level<float>& G = r->lev32[l];
        jl.add(CoefJob{G, l + 1 < ng ? r->lev32[l + 1] : G, k32(r), l + 1 < ng ? 1 : 0}, nblocks(G.ncell));
      }
      go(CHHS_K_FRAME, jl, kb_coef_restrict<DIM>, kBlock, 0, s);
    }
  }

  void norm(cudaStream_t s, bool use_cond, int mode) {
    const BatchConds* cc = use_cond ? b->d_conds : nullptr;
    JobList<NormJob> jl;
    const bool df = !b->opts.f64_residual;
    for (chhs_t* r : b->runs) {
      const Level<double>& L = r->lev[0];
      jl.add(NormJob{L, r->lev32[0], k64(r), Enqueue<DIM>::df_coefs(r), r->partials, r->st, r->norm_f64_per8},
             df ? (int)ndf_blocks(L.nx, L.ny, L.nz) : r->norm_blocks);
    }
    if (df)
      go(CHHS_K_NORM, jl, kb_norm_mixed_df<DIM>, kNdfTX * kNdfTY, 0, s, b->d_ticket, cc, mode, b->d_ticket + 1);
    else
      go(CHHS_K_NORM, jl, kb_norm_mixed<DIM>, kBlock, 0, s, b->d_ticket, cc, mode, b->d_ticket + 1);
  }

  void vcycle(cudaStream_t s) {
    const int ts = max_tail_start();
    // the options' sweeps on the finest level, the batch's coarse ones below
    // (chhs_batch_set_tuning; every run of the batch has the same)
    const chhs_t* r0 = b->runs[0];
    for (int l = 0; l < ts; ++l) pre(s, l, l == 0 ? b->opts.nu1 : r0->nu1c);
    std::vector<TailJob<float>> tails;
    for (chhs_t* r : b->runs) tails.push_back(TailJob<float>{r->tail32, k32(r), gate(r)});
    go_tail(tails, s);
    for (int l = ts - 1; l >= 0; --l) post(s, l, l == 0 ? b->opts.nu2 : r0->nu2c);
    if (vk != 1) return;
    JobList<PairJob> upd;
    for (chhs_t* r : b->runs)
      if (!Enqueue<DIM>::fused_update(r))
        upd.add(PairJob{r->lev32[0], r->lev32[0], k32(r), r->lev[0], gate(r)}, nblocks(r->lev[0].ncell));
    go(CHHS_K_FRAME, upd, kb_mixed_update, kBlock, 0, s);
  }

  // A level whose own tile grid fills the GPU several times over runs as the
  // run's own tile launch (gated), which keeps its parameters in the
  // constant bank; a batched launch would hold them in registers and
  // re-derive them per block (measured 35-50% slower on 512^2-1024^2 levels).
  // The smaller levels of all runs share one batched launch.
  static constexpr int kSoloTileBlocks = 128;  // a level of 512 x 256 cells or more
  void go_tile(int kind, const TileJob<float>& J, int blocks, cudaStream_t s) {
    if (!capture) return;
    if (counter) ++*counter;
    const int tw = b->big_tw, th = b->big_th;
    const dim3 grid((unsigned)((J.L.nx + tw - 1) / tw), (unsigned)((J.L.ny + th - 1) / th));
    timed(kind, [&] {
      pdl_grid(k_tile<float, true>, grid, b->big_tt, tile_smem_big, s, J.L, J.C, J.K, J.npass, J.halo, J.rhs,
               J.prolong, J.restrict_out, J.out, J.gate, tw, th);
    }, s);
  }
  // Side streams of the capture: the big per-run tile launches of one phase
  // run on parallel branches of the graph (one run's wave tail overlaps the
  // next run's blocks), the batched launch of the small levels beside them.
  static constexpr int kBranches = 8;
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kBranches] = {};

  void tiles(int kind, const JobList<TileJob<float>>& all, cudaStream_t s) {
    JobList<TileJob<float>> small;
    std::vector<int> big;
    for (int q = 0; q < all.njobs(); ++q) {
      const int blocks = all.start[q + 1] - all.start[q];
      if (blocks >= kSoloTileBlocks) big.push_back(q);
      else small.add(all.jobs[q], blocks);
    }
    const bool fan = capture && branch[0] && big.size() > 1;
    const int nb = fan ? std::min<int>(kBranches, (int)big.size()) : 0;
    if (fan) {
      cudaEventRecord(fork_ev, s);
      for (int q = 0; q < nb; ++q) cudaStreamWaitEvent(branch[q], fork_ev, 0);
    }
    for (size_t q = 0; q < big.size(); ++q) {
      const int jq = big[q];
      go_tile(kind, all.jobs[jq], all.start[jq + 1] - all.start[jq], fan ? branch[q % nb] : s);
    }
    go(kind, small, kb_tile<float, true>, kTileThreads, tile_smem, s);
    if (fan)
      for (int q = 0; q < nb; ++q) {
        cudaEventRecord(join_ev[q], branch[q]);
        cudaStreamWaitEvent(s, join_ev[q], 0);
      }
  }

  void pre(cudaStream_t s, int l, int nu1) {
    if (DIM == 2) {
      JobList<TileJob<float>> jl;
      const int np1 = 2 * nu1;
      for (chhs_t* r : b->runs) {
        if (l >= r->tail_start) continue;
        const Level<float>& L = r->lev32[l];
        const TileOut<float> to_copy{L.phi2, L.mu2, L.p2, L.fc1, L.fc2, L.fc3, nullptr, nullptr, nullptr};
        const int gx = (L.nx + kTileW - 1) / kTileW, gy = (L.ny + kTileH - 1) / kTileH;
        jl.add(TileJob<float>{L, r->lev32[l + 1], k32(r), to_copy, gate(r), np1, np1 + 1, l > 0 ? 1 : 0, 0, 1, gx},
               gx * gy);
      }
      tiles(l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, jl, s);
      return;
    }
    auto runs_at = [&](auto add) {
      for (chhs_t* r : b->runs)
        if (l < r->tail_start) add(r, r->lev32[l], r->lev32[l + 1]);
    };
    if (l > 0 && nu1 == 0) {
      JobList<PairJob> jl;
      runs_at([&](chhs_t* r, const Level<float>& L, const Level<float>& C) {
        jl.add(PairJob{L, C, k32(r), Level<double>{}, gate(r)}, nblocks(L.ncell));
      });
      go(CHHS_K_COARSE_RHS, jl, kb_coarse_rhs<DIM>, kBlock, 0, s);
    }
    for (int it = 0; it < nu1; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        JobList<SmoothCJob> jl;
        runs_at([&](chhs_t* r, const Level<float>& L, const Level<float>& C) {
          const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
          jl.add(SmoothCJob{L, C, Level<double>{}, k32(r), gate(r), colour, (l > 0 && it == 0) ? 1 : 0, 0},
                 (threads + kSmoothBlock - 1) / kSmoothBlock);
        });
        go(l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, jl, kb_smooth_c<DIM>, kSmoothBlock, 0, s);
      }
    JobList<PairJob> jr;
    runs_at([&](chhs_t* r, const Level<float>& L, const Level<float>& C) {
      const long long warps = rr_c_warps(DIM, L.nx, L.ny, L.nz);
      jr.add(PairJob{L, C, k32(r), Level<double>{}, gate(r)}, (int)((warps * 32 + kBlock - 1) / kBlock));
    });
    go(CHHS_K_RESTRICT, jr, kb_residual_restrict_c<DIM>, kBlock, 0, s);
  }

  void post(cudaStream_t s, int l, int nu2) {
    if (DIM == 2) {
      JobList<TileJob<float>> jl;
      const int np2 = 2 * nu2;
      for (chhs_t* r : b->runs) {
        if (l >= r->tail_start) continue;
        const Level<float>& L = r->lev32[l];
        Level<float> Lb = L;
        Lb.phi = L.phi2;
        Lb.mu = L.mu2;
        Lb.p = L.p2;
        if (l > 0) {
          Lb.fphi = L.fc1;
          Lb.fmu = L.fc2;
          Lb.fp = L.fc3;
        }
        TileOut<float> to_state{L.phi, L.mu, L.p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        if (l == 0 && Enqueue<DIM>::fused_update(r) && vk == 1) {
          to_state.phi64 = r->lev[0].phi;
          to_state.mu64 = r->lev[0].mu;
          to_state.p64 = r->lev[0].p;
        }
        const int gx = (L.nx + kTileW - 1) / kTileW, gy = (L.ny + kTileH - 1) / kTileH;
        jl.add(TileJob<float>{Lb, r->lev32[l + 1], k32(r), to_state, gate(r), np2, np2, 0, 1, 0, gx}, gx * gy);
      }
      tiles(l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, jl, s);
      return;
    }
    auto runs_at = [&](auto add) {
      for (chhs_t* r : b->runs)
        if (l < r->tail_start) add(r, r->lev32[l], r->lev32[l + 1]);
    };
    if (nu2 == 0) {
      JobList<PairJob> jl;
      runs_at([&](chhs_t* r, const Level<float>& L, const Level<float>& C) {
        jl.add(PairJob{L, C, k32(r), Level<double>{}, gate(r)}, nblocks(L.ncell));
      });
      go(CHHS_K_PROLONG, jl, kb_prolong<DIM>, kBlock, 0, s);
      return;
    }
    for (int it = 0; it < nu2; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        JobList<SmoothCJob> jl;
        const int pro = it == 0 ? (colour == 0 ? 1 : 2) : 0;
        runs_at([&](chhs_t* r, const Level<float>& L, const Level<float>& C) {
          const bool upd = l == 0 && Enqueue<DIM>::fused_update(r) && vk == 1 && it == nu2 - 1 && colour == 1;
          const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
          jl.add(SmoothCJob{L, C, upd ? r->lev[0] : Level<double>{}, k32(r), gate(r), colour, 0, pro},
                 (threads + kSmoothBlock - 1) / kSmoothBlock);
        });
        go(l == 0 ? CHHS_K_SMOOTH_FINEST : CHHS_K_SMOOTH, jl, kb_smooth_c<DIM>, kSmoothBlock, 0, s);
      }
  }

  void advance(cudaStream_t s) {
    JobList<AdvanceJob> jl;
    for (chhs_t* r : b->runs) jl.add(AdvanceJob{r->lev[0], r->phimm1, r->st}, nblocks(r->lev[0].ncell));
    go(CHHS_K_FRAME, jl, kb_advance, kBlock, 0, s);
  }

  // Plan: lay out every table in emission order (no CUDA calls).
  void plan() {
    capture = false;
    setup(nullptr);
    coefs(nullptr);
    norm(nullptr, false, 0);
    for (vk = n_if() + 1; vk >= 1; --vk) {
      vstart[vk] = offs.size();
      vcycle(nullptr);
    }
    vk = 1;
    vstart[0] = offs.size();
    norm(nullptr, false, 1);
    advance(nullptr);
  }

  // Shared memory of the batched tile and tail launches, opted in (only ever raised).
  chhs_status prepare() {
    int dev = 0, optin = 0;
    BCU(cudaGetDevice(&dev));
    BCU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (chhs_t* r : b->runs) tail_smem = std::max(tail_smem, Enqueue<DIM>::template tail_bytes<float, true>(r->tail32));
    if (DIM == 2) {
      const int halo = 2 * std::max(std::max(b->opts.nu1, b->opts.nu2), std::max(b->runs[0]->nu1c, b->runs[0]->nu2c)) + 1;
      tile_smem = tile_smem_bytes(halo, tile_nfields<true>(), sizeof(float));
      tile_smem_big = tile_smem_bytes(halo, tile_nfields<true>(), sizeof(float), b->big_tw, b->big_th);
    }
    auto raise_to = [&](const void* fn, size_t dyn) -> chhs_status {
      cudaFuncAttributes fa;
      BCU(cudaFuncGetAttributes(&fa, fn));
      if (dyn + fa.sharedSizeBytes > (size_t)optin)
        return bfail(b, CHHS_ERR_INVALID_ARG, "a run's coarse tail or tiles need more shared memory than a block has");
      if ((size_t)fa.maxDynamicSharedSizeBytes < dyn)
        BCU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      return CHHS_OK;
    };
    chhs_status st = raise_to(reinterpret_cast<const void*>(kb_tail<float, DIM, true>), tail_smem);
    if (st != CHHS_OK) return st;
    if (DIM == 2) {
      st = raise_to(reinterpret_cast<const void*>(kb_tile<float, true>), tile_smem);
      if (st != CHHS_OK) return st;
      st = raise_to(reinterpret_cast<const void*>(k_tile<float, true>), std::max(tile_smem, tile_smem_big));
      if (st != CHHS_OK) return st;
    }
    return CHHS_OK;
  }

  // Capture the step graph (the structure of a single run's build_graph).
  chhs_status build() {
    chhs_status ps = prepare();
    if (ps != CHHS_OK) return ps;
    plan();
    BCU(cudaMalloc(&b->tables, std::max<size_t>(buf.size(), 256)));
    BCU(cudaMemcpy(b->tables, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    capture = true;
    cur = 0;
    struct CaptureRes {
      cudaStream_t s[4 + kBranches] = {};
      cudaEvent_t e[3 + kBranches] = {};
      ~CaptureRes() {
        for (int q : {3 + kBranches, 1, 0}) {  // the IF bodies', the loop body's, the step's capture
          cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
          if (s[q] && cudaStreamIsCapturing(s[q], &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(s[q], &g);
            if (q == 0 && g) cudaGraphDestroy(g);
          }
        }
        for (cudaEvent_t ev : e)
          if (ev) cudaEventDestroy(ev);
        for (cudaStream_t st : s)
          if (st) cudaStreamDestroy(st);
        cudaGetLastError();
      }
    } res;
    for (int q = 0; q < 4 + kBranches; ++q) BCU(cudaStreamCreateWithFlags(&res.s[q], cudaStreamNonBlocking));
    for (int q = 0; q < 3 + kBranches; ++q) BCU(cudaEventCreateWithFlags(&res.e[q], cudaEventDisableTiming));
    cudaStream_t cs = res.s[0], cs2 = res.s[1], cs3 = res.s[2], cs4 = res.s[3 + kBranches];
    for (int q = 0; q < kBranches; ++q) {
      branch[q] = res.s[3 + q];
      join_ev[q] = res.e[3 + q];
    }
    fork_ev = res.e[2];
    int n_frame = 0, n_v = 0, n_other = 0;
    BCU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    counter = &n_frame;
    setup(cs);
    BCU(cudaEventRecord(res.e[0], cs));
    BCU(cudaStreamWaitEvent(cs3, res.e[0], 0));
    coefs(cs3);
    BCU(cudaEventRecord(res.e[1], cs3));
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    BCU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle cond;
    BCU(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    norm(cs, true, 0);
    BCU(cudaStreamWaitEvent(cs, res.e[1], 0));
    BCU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    BCU(cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp));
    BCU(cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BCU(cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // the loop body as in a single run's graph: IF (some run takes a 4th
    // V-cycle) V-cycle 4; ... IF (a 2nd) V-cycle 2; V-cycle 1 with the
    // update; the norms, whose last report sets the conditions
    BatchConds hc{};
    hc.loop = cond;
    hc.nif = n_if();
    for (vk = n_if() + 1; vk >= 2; --vk) {
      cudaGraph_t bg = nullptr;
      BCU(cudaStreamGetCaptureInfo(cs2, &cst, nullptr, &bg, &deps, nullptr, &ndeps));
      BCU(cudaGraphConditionalHandleCreate(&hc.cif[vk - 2], bg, 0, cudaGraphCondAssignDefault));
      cudaGraphNodeParams ip{};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hc.cif[vk - 2];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t ifn;
      BCU(cudaGraphAddNode(&ifn, bg, deps, nullptr, ndeps, &ip));
      BCU(cudaStreamUpdateCaptureDependencies(cs2, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
      cudaGraph_t ib = ip.conditional.phGraph_out[0];
      BCU(cudaStreamBeginCaptureToGraph(cs4, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      counter = &n_other;
      vcycle(cs4);
      BCU(cudaStreamEndCapture(cs4, &ib));
    }
    vk = 1;
    counter = &n_v;
    vcycle(cs2);
    counter = &n_other;
    norm(cs2, true, 1);
    BCU(cudaStreamEndCapture(cs2, &body));
    counter = &n_frame;
    advance(cs);
    counter = nullptr;
    BCU(cudaStreamEndCapture(cs, &b->graph));
    for (int q = 0; q < kBranches; ++q) branch[q] = nullptr;
    BCU(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->launches_per_v = n_v;
    b->launches_per_step = n_frame;
    BCU(cudaMemcpy(b->d_conds, &hc, sizeof(hc), cudaMemcpyHostToDevice));
    return CHHS_OK;
  }

  // One step launched kernel by kernel with events (the loop decided on the
  // host from the "any run iterating" flag of the batched norm).
  chhs_status profile(Prof* p) {
    plan();  // the same emission order as the captured graph
    capture = true;
    cur = 0;
    prof = p;
    cudaStream_t s = b->stream;
    setup(s);
    coefs(s);
    norm(s, false, 0);
    for (int v = 0;; ++v) {
      unsigned int any[kMaxInner] = {};  // some run iterating, taking a 2nd, 3rd, ... V-cycle
      BCU(cudaMemcpyAsync(any, b->d_ticket + 1, sizeof(any), cudaMemcpyDeviceToHost, s));
      BCU(cudaStreamSynchronize(s));
      if (!any[0]) break;
      for (vk = n_if() + 1; vk >= 1; --vk) {
        if (vk > 1 && !any[vk - 1]) continue;
        cur = vstart[vk];
        vcycle(s);
      }
      vk = 1;
      cur = vstart[0];
      norm(s, false, 1);
    }
    cur = offs.size() - 2;  // the advance's jobs and prefix sum come last
    advance(s);
    prof = nullptr;
    BCU(cudaGetLastError());
    BCU(cudaStreamSynchronize(s));
    return CHHS_OK;
  }
};

void batch_free(chhs_batch_t* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (chhs_t* r : b->runs) destroy_handle(r);
  if (b->tables) cudaFree(b->tables);
  if (b->arena) cudaFree(b->arena);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Bytes of the batch's own bookkeeping after the runs' hierarchies.
size_t batch_misc_bytes(int nruns) {
  return align_up(sizeof(DevState*) * nruns) + align_up((1 + kMaxInner) * sizeof(unsigned int)) +
         align_up(sizeof(BatchConds)) +
         align_up((2 * sizeof(int) + sizeof(double)) * nruns);
}

bool batch_args_ok(int nruns, const chhs_run_desc* runs, const chhs_opts& o) {
  if (nruns < 1 || !runs || !valid_opts(o) || o.precision != 1) return false;
  for (int r = 0; r < nruns; ++r) {
    const chhs_run_desc& d = runs[r];
    if (d.dim != runs[0].dim || !valid_problem(d.dim, d.n, d.h, d.eps, d.gamma, d.dt)) return false;
  }
  return true;
}

size_t batch_bytes(int nruns, const chhs_run_desc* runs, const chhs_opts& o, std::vector<size_t>* offs) {
  size_t total = 0;
  for (int r = 0; r < nruns; ++r) {
    const int nn[3] = {runs[r].n[0], runs[r].n[1], runs[r].dim == 3 ? runs[r].n[2] : 1};
    if (offs) offs->push_back(total);
    total += align_up(make_layout(runs[r].dim, nn, o.coarsest, o.precision).total);
  }
  return total + batch_misc_bytes(nruns);
}

}  // namespace

extern "C" {

size_t chhs_batch_workspace_bytes(int nruns, const chhs_run_desc* runs, const chhs_opts* opts) {
  chhs_opts o;
  chhs_default_opts(&o);
  o.precision = 1;
  if (opts) o = *opts;
  if (!batch_args_ok(nruns, runs, o)) return 0;
  return batch_bytes(nruns, runs, o, nullptr);
}

chhs_status chhs_batch_create(int nruns, const chhs_run_desc* runs, const chhs_opts* opts, void* cuda_stream,
                              chhs_batch_t** out) {
  if (!out) return CHHS_ERR_INVALID_ARG;
  *out = nullptr;
  chhs_opts o;
  chhs_default_opts(&o);
  o.precision = 1;
  if (opts) o = *opts;
  if (!batch_args_ok(nruns, runs, o)) return CHHS_ERR_INVALID_ARG;
  chhs_batch_t* b = new (std::nothrow) chhs_batch_t();
  if (!b) return CHHS_ERR_OOM;
  b->dim = runs[0].dim;
  b->nruns = nruns;
  b->opts = o;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return CHHS_ERR_CUDA;
  } else {
    b->own_stream = true;
  }
  std::vector<size_t> offs;
  const size_t total = batch_bytes(nruns, runs, o, &offs);
  if (cudaMalloc(&b->arena, total) != cudaSuccess) {
    cudaGetLastError();
    b->arena = nullptr;
    batch_free(b);
    return CHHS_ERR_OOM;
  }
  for (int r = 0; r < nruns; ++r) {
    const chhs_run_desc& d = runs[r];
    chhs_t* run = nullptr;
    const int nn[3] = {d.n[0], d.n[1], d.dim == 3 ? d.n[2] : 1};
    const size_t need = align_up(make_layout(d.dim, nn, o.coarsest, o.precision).total);
    chhs_status s = create_impl(d.dim, d.n, d.h, d.eps, d.gamma, d.dt, &o, b->stream, b->arena + offs[r], need, &run,
                                true);
    if (s != CHHS_OK) {
      batch_free(b);
      return s;
    }
    b->runs.push_back(run);
  }
  char* misc = b->arena + (total - batch_misc_bytes(nruns));
  b->d_sts = reinterpret_cast<DevState**>(misc);
  misc += align_up(sizeof(DevState*) * nruns);
  b->d_ticket = reinterpret_cast<unsigned int*>(misc);  // ticket, then the kMaxInner "any run" flags
  misc += align_up((1 + kMaxInner) * sizeof(unsigned int));
  b->d_conds = reinterpret_cast<BatchConds*>(misc);
  misc += align_up(sizeof(BatchConds));
  b->d_out = reinterpret_cast<int*>(misc);
  std::vector<DevState*> sts;
  for (chhs_t* r : b->runs) sts.push_back(r->st);
  chhs_status s = CHHS_OK;
  const size_t out_bytes = (2 * sizeof(int) + sizeof(double)) * nruns;
  if (cudaMemcpy(b->d_sts, sts.data(), sizeof(DevState*) * nruns, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_ticket, 0, (1 + kMaxInner) * sizeof(unsigned int)) != cudaSuccess ||
      cudaMallocHost(&b->h_out, out_bytes) != cudaSuccess)
    s = CHHS_ERR_CUDA;
  if (s == CHHS_OK) {
    if (b->dim == 2) {
      BatchStep<2> bs{b};
      s = bs.build();
    } else {
      BatchStep<3> bs{b};
      s = bs.build();
    }
  }
  if (s == CHHS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) s = CHHS_ERR_CUDA;
  if (s != CHHS_OK) {
    cudaGetLastError();
    batch_free(b);
    return s;
  }
  *out = b;
  return CHHS_OK;
}

int chhs_batch_size(const chhs_batch_t* b) { return b ? b->nruns : 0; }

chhs_t* chhs_batch_run(chhs_batch_t* b, int r) {
  if (!b || r < 0 || r >= b->nruns) return nullptr;
  return b->runs[r];
}

chhs_status chhs_batch_step(chhs_batch_t* b, int nsteps, int* status_out, int* vcycles_out, double* resid_out) {
  if (!b) return CHHS_ERR_INVALID_ARG;
  if (nsteps < 0) return bfail(b, CHHS_ERR_INVALID_ARG, "nsteps < 0");
  b->err.clear();
  const int n = b->nruns;
  const double tol_max = tol_max_of(b->opts);
  kb_reset<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_sts, n, b->opts.tol, tol_max, b->opts.max_v,
                                                    b->opts.max_inner);
  BCU(cudaGetLastError());
  for (int k = 0; k < nsteps; ++k) BCU(cudaGraphLaunch(b->exec, b->stream));
  int* d_status = b->d_out;
  int* d_v = d_status + n;
  double* d_res = reinterpret_cast<double*>(reinterpret_cast<char*>(b->d_out) + 2 * sizeof(int) * n);
  kb_gather<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_sts, n, d_status, d_v, d_res);
  BCU(cudaGetLastError());
  const size_t out_bytes = (2 * sizeof(int) + sizeof(double)) * n;
  BCU(cudaMemcpyAsync(b->h_out, b->d_out, out_bytes, cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  const int* hs = reinterpret_cast<const int*>(b->h_out);
  const int* hv = hs + n;
  const double* hr = reinterpret_cast<const double*>(b->h_out + 2 * sizeof(int) * n);
  chhs_status worst = CHHS_OK;
  for (int r = 0; r < n; ++r) {
    if (status_out) status_out[r] = hs[r];
    if (vcycles_out) vcycles_out[r] = hv[r];
    if (resid_out) resid_out[r] = hr[r];
    if (hs[r] != 0 && worst == CHHS_OK) {
      worst = (chhs_status)hs[r];
      char m[96];
      snprintf(m, sizeof m, "run %d: %s (residual %.3e)", r,
               hs[r] == CHHS_ERR_NOT_CONVERGED ? "not converged" : "diverged", hr[r]);
      b->err = m;
    }
  }
  return worst;
}

chhs_status chhs_batch_launch_counts(const chhs_batch_t* b, int* per_vcycle, int* per_step) {
  if (!b || !per_vcycle || !per_step) return CHHS_ERR_INVALID_ARG;
  *per_vcycle = b->launches_per_v;
  *per_step = b->launches_per_step;
  return CHHS_OK;
}

}  // extern "C"

namespace {

// Apply a tuning to every run of the batch and rebuild its step graph.
chhs_status batch_apply(chhs_batch_t* b, int tail_cells, int nu1c, int nu2c, int norm_f64_per8, int tw, int th,
                        int tt) {
  BCU(cudaStreamSynchronize(b->stream));
  b->big_tw = tw;
  b->big_th = th;
  b->big_tt = tt;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->tables) cudaFree(b->tables);
  b->exec = nullptr;
  b->graph = nullptr;
  b->tables = nullptr;
  for (chhs_t* r : b->runs) {
    r->tail_cells = tail_cells;
    r->nu1c = nu1c;
    r->nu2c = nu2c;
    r->norm_f64_per8 = norm_f64_per8;
    place_tail(r);
  }
  chhs_status s;
  if (b->dim == 2) {
    BatchStep<2> bs{b};
    s = bs.build();
  } else {
    BatchStep<3> bs{b};
    s = bs.build();
  }
  if (s == CHHS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) s = CHHS_ERR_CUDA;
  cudaGetLastError();
  return s;
}

bool batch_tuning_ok(const chhs_tuning* t) {
  return t && t->tail_cells >= 1 && t->coarse_nu1 >= 0 && t->coarse_nu2 >= 0 &&
         t->coarse_nu1 + t->coarse_nu2 >= 1 && t->norm_f64_per8 >= 0 && t->norm_f64_per8 <= 8 &&
         t->tile_threads >= 32 && t->tile_threads <= 1024 && t->tile_threads % 32 == 0 && t->tile_w >= 2 &&
         t->tile_h >= 2 && t->tile_w % 2 == 0 && t->tile_h % 2 == 0 && t->tile_w * t->tile_h <= 4096;
}

}  // namespace

extern "C" {

chhs_status chhs_batch_set_tuning(chhs_batch_t* b, const chhs_tuning* t) {
  if (!b) return CHHS_ERR_INVALID_ARG;
  if (!batch_tuning_ok(t)) return bfail(b, CHHS_ERR_INVALID_ARG, "invalid tuning");
  b->err.clear();
  const chhs_t* r0 = b->runs[0];
  const int keep[7] = {r0->tail_cells, r0->nu1c, r0->nu2c, r0->norm_f64_per8, b->big_tw, b->big_th, b->big_tt};
  chhs_status s = batch_apply(b, t->tail_cells, t->coarse_nu1, t->coarse_nu2, t->norm_f64_per8, t->tile_w, t->tile_h,
                              t->tile_threads);
  if (s == CHHS_OK) return CHHS_OK;
  const std::string why = b->err;
  if (batch_apply(b, keep[0], keep[1], keep[2], keep[3], keep[4], keep[5], keep[6]) != CHHS_OK)
    return bfail(b, CHHS_ERR_CUDA, why);
  return bfail(b, s == CHHS_ERR_CUDA ? CHHS_ERR_CUDA : CHHS_ERR_INVALID_ARG, why);
}

chhs_status chhs_batch_autotune(chhs_batch_t* b, int trial_steps, chhs_tuning* out) {
  if (!b || trial_steps < 1) return bfail(b, CHHS_ERR_INVALID_ARG, "bad argument");
  b->err.clear();
  // every run's state (phi^m, phi^{m-1}, mu, p), restored after each trial
  size_t total = 0;
  for (const chhs_t* r : b->runs) total += 4 * (size_t)r->ncell();
  double* keep = nullptr;
  if (cudaMalloc(&keep, sizeof(double) * total) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, CHHS_ERR_OOM, "no room for the saved states");
  }
  auto copy_states = [&](bool save) -> bool {
    size_t off = 0;
    for (chhs_t* r : b->runs) {
      const Level<double>& F = r->lev[0];
      double* st[4] = {F.phim, r->phimm1, F.mu, F.p};
      const size_t bytes = sizeof(double) * r->ncell();
      for (double* a : st) {
        if (cudaMemcpyAsync(save ? keep + off : a, save ? a : keep + off, bytes, cudaMemcpyDeviceToDevice,
                            b->stream) != cudaSuccess)
          return false;
        off += r->ncell();
      }
    }
    return cudaStreamSynchronize(b->stream) == cudaSuccess;
  };
  struct Cand {
    int tc, n1, n2, tw, th, tt;
  };
  const chhs_t* r0 = b->runs[0];
  const Cand orig{r0->tail_cells, r0->nu1c, r0->nu2c, b->big_tw, b->big_th, b->big_tt};
  std::vector<Cand> cands;
  std::vector<std::pair<int, int>> coarse = {{b->opts.nu1, b->opts.nu2}};
  if (b->opts.nu1 > 1 && b->opts.nu2 > 1) coarse.push_back({1, 1});
  // 2D: the tile shape of the per-run launches of large levels as well
  const int shapes2[3][3] = {{kTileW, kTileH, kTileThreads}, {32, 32, 512}, {64, 16, 512}};
  const int nshapes = b->dim == 2 ? 3 : 1;
  for (const auto& cn : coarse)
    for (int tc : {b->dim == 2 ? 256 : 64, b->dim == 2 ? 1024 : 512, 4096})
      for (int q = 0; q < nshapes; ++q)
        cands.push_back({tc, cn.first, cn.second, shapes2[q][0], shapes2[q][1], shapes2[q][2]});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  chhs_status s = CHHS_OK;
  float best_ms = -1.f;
  Cand best = orig;
  if (!copy_states(true) || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    s = CHHS_ERR_CUDA;
  for (size_t q = 0; s == CHHS_OK && q < cands.size(); ++q) {
    const Cand& c = cands[q];
    if (batch_apply(b, c.tc, c.n1, c.n2, r0->norm_f64_per8, c.tw, c.th, c.tt) != CHHS_OK) continue;  // e.g. a tail too big
    // one untimed step (the new graph's first launch), then the timed ones,
    // each from the saved state
    bool ok = copy_states(false) && chhs_batch_step(b, 1, nullptr, nullptr, nullptr) == CHHS_OK && copy_states(false);
    if (!ok) continue;
    const int n = b->nruns;
    kb_reset<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_sts, n, b->opts.tol, tol_max_of(b->opts), b->opts.max_v,
                                                      b->opts.max_inner);
    cudaEventRecord(e0, b->stream);
    for (int k = 0; k < trial_steps; ++k) cudaGraphLaunch(b->exec, b->stream);
    cudaEventRecord(e1, b->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      s = CHHS_ERR_CUDA;
      break;
    }
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  if (s == CHHS_OK && batch_apply(b, best.tc, best.n1, best.n2, r0->norm_f64_per8, best.tw, best.th, best.tt) != CHHS_OK) {
    best_ms = -1.f;  // the fastest could not be rebuilt: back to the original setting
    if (batch_apply(b, orig.tc, orig.n1, orig.n2, r0->norm_f64_per8, orig.tw, orig.th, orig.tt) != CHHS_OK)
      s = CHHS_ERR_CUDA;
  }
  if (s == CHHS_OK && !copy_states(false)) s = CHHS_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(keep);
  cudaGetLastError();
  if (s != CHHS_OK) return bfail(b, s, "autotune failed");
  b->err.clear();  // a trial's failed candidate left its message
  if (out) {
    const chhs_t* r = b->runs[0];
    out->tail_cells = r->tail_cells;
    out->split_threads = r->split_threads;
    out->tile_threads = b->big_tt;
    out->coarse_nu1 = r->nu1c;
    out->coarse_nu2 = r->nu2c;
    out->tile_w = b->big_tw;
    out->tile_h = b->big_th;
    out->norm_f64_per8 = r->norm_f64_per8;
    out->small_tile_w = kTileW;
    out->small_tile_h = kTileH;
    out->small_tile_threads = kTileThreads;
    out->quad_passes = 0;
    out->ms_per_step = best_ms < 0.f ? -1.0 : best_ms / trial_steps;
  }
  return CHHS_OK;
}

chhs_status chhs_batch_profile_step(chhs_batch_t* b, double* ms_out, long long* launches_out) {
  if (!b || !ms_out || !launches_out) return bfail(b, CHHS_ERR_INVALID_ARG, "NULL argument");
  b->err.clear();
  const int n = b->nruns;
  kb_reset<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_sts, n, b->opts.tol, tol_max_of(b->opts), b->opts.max_v,
                                                    b->opts.max_inner);
  BCU(cudaGetLastError());
  Prof prof;
  chhs_status s;
  if (b->dim == 2) {
    BatchStep<2> bs{b};
    bs.prepare();
    s = bs.profile(&prof);
  } else {
    BatchStep<3> bs{b};
    bs.prepare();
    s = bs.profile(&prof);
  }
  if (s != CHHS_OK) return s;
  for (size_t q = 0; q < prof.kind.size(); ++q) {
    float ms = 0.f;
    BCU(cudaEventElapsedTime(&ms, prof.ev[2 * q], prof.ev[2 * q + 1]));
    ms_out[prof.kind[q]] += ms;
    launches_out[prof.kind[q]] += 1;
  }
  return CHHS_OK;
}

const char* chhs_batch_last_error(const chhs_batch_t* b) { return b ? b->err.c_str() : "NULL batch"; }

void chhs_batch_destroy(chhs_batch_t* b) { batch_free(b); }

}  // extern "C"
