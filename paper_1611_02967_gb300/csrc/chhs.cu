// chhs.cu -- host side of the C ABI declared in include/chhs.h: argument
// checks, the device hierarchy in one arena, and the per-step CUDA graph.
//
// One time step is one CUDA graph launch:
//   setup (phi*, right-hand sides, initial guess)     Eq. 2.4 and 2.5-2.7
//   restrict phi^m, phi* to every coarse level
//   stopping norm -> while-loop condition
//   WHILE (norm > tol and V < max_v):                 Section 5 preamble
//       V(nu1, nu2)-cycle; stopping norm -> condition
//   mean of p; accept the step (rotate phi^m, phi^{m-1})
// The loop is a conditional graph node whose condition a device kernel sets,
// so a step needs no host round trip; chhs_step(n) launches the graph n times
// and reads the device status once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/chhs.h"
#include "chhs_kernels.cuh"

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

// phi mu p fphi fmu fp phim phis phi0 mu0 p0, ax ay Mx My, sM sa, cAe cCD cG (+ az Mz in 3D)
constexpr int kBaseFields = 11;
int level_fields(int dim) { return kBaseFields + (dim == 3 ? 11 : 9); }

// Levels with at most this many cells run inside the one-block tail kernel.
// In double precision one SM does 2 FMA per clock, so only the tiniest levels
// (8 x 8, 4 x 4 x 4) are cheaper there than as grid-wide launches.
constexpr int kTailCellsF64 = 64;

struct Layout {
  std::vector<Shape> shapes;
  size_t state_off, partial_off, phimm1_off;
  std::vector<size_t> level_off;  // start of each level's field arrays
  size_t total;
  int nparts;  // partial-sum slots (blocks of the finest grid)
};

Layout make_layout(int dim, const int n[3], int coarsest) {
  Layout L;
  L.shapes = level_shapes(dim, n, coarsest);
  size_t off = 0;
  L.state_off = off;
  off += align_up(sizeof(DevState));
  int nf = L.shapes[0].n[0] * L.shapes[0].n[1] * L.shapes[0].n[2];
  L.nparts = nblocks(nf);
  L.partial_off = off;
  off += align_up(sizeof(double) * 6 * (size_t)L.nparts);
  L.phimm1_off = off;
  off += align_up(sizeof(double) * (size_t)nf);
  for (const Shape& s : L.shapes) {
    size_t nc = (size_t)s.n[0] * s.n[1] * s.n[2];
    L.level_off.push_back(off);
    off += level_fields(dim) * align_up(sizeof(double) * nc);
  }
  L.total = off;
  return L;
}

bool valid_opts(const chhs_opts& o) {
  return o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 >= 1 && o.max_v >= 1 && o.coarsest >= 1 &&
         o.tol > 0 && (o.precision == 0);
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
  std::vector<Level<double>> lev;
  int tail_start = 0;   // first level run by the one-block tail kernel
  Tail<double> tail{};  // its levels
  double* phimm1 = nullptr;
  DevState* st = nullptr;
  double* partials = nullptr;
  DevState* host_st = nullptr;  // pinned mirror
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches_per_v = 0, launches_per_step = 0;
  int* counter = nullptr;  // counts launches while the graph is captured
  Prof* prof = nullptr;  // per-launch events while profiling
  std::string err;
  int ncell() const { return n[0] * n[1] * n[2]; }
};

namespace {

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

// Cells of colour 0 ((i+j+k) even) in a box whose corner cell is even.
double colour_cells(const Level<double>& L, int colour) {
  double n = L.ncell;
  bool odd = (L.ncell & 1) != 0;
  return colour == 0 ? (odd ? (n + 1) / 2 : n / 2) : (odd ? (n - 1) / 2 : n / 2);
}

template <int DIM>
struct Enqueue {
  static Coefs<double> coefs(const chhs_t* run) {
    return Coefs<double>{run->dt, run->gamma, 0.75 * run->eps * run->eps};
  }

  // sweeps red-black sweeps; with rhs the first one also completes the FAS
  // right-hand side of this (coarse) level.
  static void smooth(chhs_t* run, cudaStream_t s, const Level<double>& L, int sweeps, bool rhs) {
    const Coefs<double> K = coefs(run);
    const int threads = ((L.nx + 1) / 2) * L.ny * L.nz;
    const int blocks = (threads + kSmoothBlock - 1) / kSmoothBlock;
    for (int it = 0; it < sweeps; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        const int with_rhs = (rhs && it == 0) ? 1 : 0;
        launch(run, s, CHHS_K_SMOOTH, colour_cells(L, colour), [&] {
          k_smooth<double, DIM, false><<<blocks, kSmoothBlock, 0, s>>>(L, K, colour, with_rhs);
        });
      }
  }

  static void vcycle(chhs_t* run, cudaStream_t s, int l) {
    const Coefs<double> K = coefs(run);
    const Level<double>& L = run->lev[l];
    if (l == run->tail_start) {
      launch(run, s, CHHS_K_COARSEST, 1.0, [&] {
        k_tail<double, DIM, false><<<1, kTailThreads, 0, s>>>(run->tail, K);
      });
      return;
    }
    const Level<double>& C = run->lev[l + 1];
    const bool rhs = l > 0;
    if (rhs && run->opts.nu1 == 0)
      launch(run, s, CHHS_K_COARSE_RHS, L.ncell, [&] {
        k_coarse_rhs<double, DIM, false><<<nblocks(L.ncell), kBlock, 0, s>>>(L, K);
      });
    smooth(run, s, L, run->opts.nu1, rhs && run->opts.nu1 > 0);
    constexpr int TX = DIM == 3 ? 8 : 16;
    const long long tiles = (long long)((L.nx + TX - 1) / TX) * (L.ny / 2) * (DIM == 3 ? L.nz / 2 : 1);
    const int rblocks = (int)((tiles * 32 + kBlock - 1) / kBlock);
    launch(run, s, CHHS_K_RESTRICT, L.ncell, [&] {
      k_residual_restrict<double, DIM, false><<<rblocks, kBlock, 0, s>>>(L, C, K);
    });
    vcycle(run, s, l + 1);
    launch(run, s, CHHS_K_PROLONG, L.ncell, [&] {
      k_prolong<double, DIM><<<nblocks(L.ncell), kBlock, 0, s>>>(L, C);
    });
    smooth(run, s, L, run->opts.nu2, false);
  }

  static void norm(chhs_t* run, cudaStream_t s, cudaGraphConditionalHandle cond, int mode, int use_cond) {
    const Coefs<double> K = coefs(run);
    const Level<double>& L = run->lev[0];
    launch(run, s, CHHS_K_NORM, L.ncell, [&] {
      k_norm<double, DIM><<<nblocks(L.ncell), kBlock, 0, s>>>(L, K, run->partials, run->st, cond, mode,
                                                              use_cond);
    });
  }

  static void frame_head(chhs_t* run, cudaStream_t s) {
    const Level<double>& F = run->lev[0];
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      k_setup<DIM><<<nblocks(F.ncell), kBlock, 0, s>>>(F, run->phimm1, run->eps * run->eps, run->st);
    });
    for (size_t l = 1; l < run->lev.size(); ++l)
      launch(run, s, CHHS_K_FRAME, 1.0, [&] {
        k_restrict_coef<double, DIM><<<nblocks(run->lev[l].ncell), kBlock, 0, s>>>(run->lev[l - 1],
                                                                                  run->lev[l]);
      });
    const Coefs<double> K = coefs(run);
    for (size_t l = 0; l < run->lev.size(); ++l)
      launch(run, s, CHHS_K_FRAME, 1.0, [&] {
        k_coef<double, DIM><<<nblocks(run->lev[l].ncell), kBlock, 0, s>>>(run->lev[l], K);
      });
  }

  static void frame_tail(chhs_t* run, cudaStream_t s) {
    const Level<double>& F = run->lev[0];
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      k_sum_partial<<<nblocks(F.ncell), kBlock, 0, s>>>(F.p, F.ncell, run->partials);
    });
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      k_mean_finish<<<1, 1024, 0, s>>>(run->partials, nblocks(F.ncell), F.ncell, run->st);
    });
    launch(run, s, CHHS_K_FRAME, 1.0, [&] {
      k_advance<<<nblocks(F.ncell), kBlock, 0, s>>>(F, run->phimm1, run->st);
    });
  }

  static chhs_status build_graph(chhs_t* run) {
    cudaStream_t cs = nullptr, cs2 = nullptr;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
    int n_frame = 0, n_v = 0;
    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    run->counter = &n_frame;
    frame_head(run, cs);
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cst;
    CU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle cond;
    CU(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    norm(run, cs, cond, 0, 1);
    CU(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    CU(cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp));
    CU(cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    run->counter = &n_v;
    vcycle(run, cs2, 0);
    norm(run, cs2, cond, 1, 1);
    CU(cudaStreamEndCapture(cs2, &body));
    run->counter = &n_frame;
    frame_tail(run, cs);
    run->counter = nullptr;
    CU(cudaStreamEndCapture(cs, &run->graph));
    CU(cudaGraphInstantiate(&run->exec, run->graph, 0));
    CU(cudaStreamDestroy(cs2));
    CU(cudaStreamDestroy(cs));
    run->launches_per_v = n_v;
    run->launches_per_step = n_frame;
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
      vcycle(run, s, 0);
      norm(run, s, 0, 1, 0);
    }
    frame_tail(run, s);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
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

__global__ void k_reset_call(DevState* st, double tol, int max_v) {
  st->failed = 0;
  st->vtotal = 0;
  st->steps_done = 0;
  st->tol = tol;
  st->max_v = max_v;
}

chhs_status setup_handle(chhs_t* run) {
  const Layout& Lo = run->layout;
  run->st = reinterpret_cast<DevState*>(run->arena + Lo.state_off);
  run->partials = reinterpret_cast<double*>(run->arena + Lo.partial_off);
  run->phimm1 = reinterpret_cast<double*>(run->arena + Lo.phimm1_off);
  double hl = run->h;
  for (size_t l = 0; l < Lo.shapes.size(); ++l) {
    const Shape& s = Lo.shapes[l];
    size_t nc = (size_t)s.n[0] * s.n[1] * s.n[2];
    size_t stride = align_up(sizeof(double) * nc);
    char* base = run->arena + Lo.level_off[l];
    const int nf = level_fields(run->dim);
    double* f[kBaseFields + 11];
    for (int q = 0; q < nf; ++q) f[q] = reinterpret_cast<double*>(base + q * stride);
    Level<double> L;
    L.phi = f[0]; L.mu = f[1]; L.p = f[2];
    L.fphi = f[3]; L.fmu = f[4]; L.fp = f[5];
    L.phim = f[6]; L.phis = f[7];
    L.phi0 = f[8]; L.mu0 = f[9]; L.p0 = f[10];
    L.ax = f[11]; L.ay = f[12]; L.Mx = f[13]; L.My = f[14];
    L.sM = f[15]; L.sa = f[16];
    L.cAe = f[17]; L.cCD = f[18]; L.cG = f[19];
    L.az = run->dim == 3 ? f[20] : nullptr;
    L.Mz = run->dim == 3 ? f[21] : nullptr;
    L.phib = nullptr;
    L.nx = s.n[0]; L.ny = s.n[1]; L.nz = s.n[2];
    L.ncell = (int)nc;
    L.ih2 = 1.0 / (hl * hl);
    L.h2 = hl * hl;
    L.sih2 = run->dt * L.ih2;
    L.e34ih2 = 0.75 * run->eps * run->eps * L.ih2;
    run->lev.push_back(L);
    hl *= 2.0;
  }
  const int nl = (int)run->lev.size();
  run->tail_start = nl - 1;
  while (run->tail_start > 0 && run->lev[run->tail_start - 1].ncell <= kTailCellsF64 &&
         nl - (run->tail_start - 1) <= kTailMaxLevels)
    --run->tail_start;
  run->tail.n = nl - run->tail_start;
  for (int l = run->tail_start; l < nl; ++l) run->tail.lev[l - run->tail_start] = run->lev[l];
  run->tail.nu1 = run->opts.nu1;
  run->tail.nu2 = run->opts.nu2;
  run->tail.top_rhs = run->tail_start > 0 ? 1 : 0;
  CU(cudaMemsetAsync(run->arena, 0, Lo.total, run->stream));
  CU(cudaMallocHost(&run->host_st, sizeof(DevState)));
  memset(run->host_st, 0, sizeof(DevState));
  chhs_status s = run->dim == 2 ? Enqueue<2>::build_graph(run) : Enqueue<3>::build_graph(run);
  if (s != CHHS_OK) return s;
  CU(cudaStreamSynchronize(run->stream));
  return CHHS_OK;
}

chhs_status create_impl(int dim, const int n[3], double h, double eps, double gamma, double dt,
                        const chhs_opts* opts, void* cuda_stream, void* arena, size_t arena_bytes,
                        chhs_t** out) {
  if (!out) return CHHS_ERR_INVALID_ARG;
  *out = nullptr;
  chhs_opts o;
  chhs_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_problem(dim, n, h, eps, gamma, dt) || !valid_opts(o)) return CHHS_ERR_INVALID_ARG;
  chhs_t* run = new (std::nothrow) chhs_t();
  if (!run) return CHHS_ERR_OOM;
  run->dim = dim;
  for (int a = 0; a < 3; ++a) run->n[a] = (a < dim) ? n[a] : 1;
  run->h = h; run->eps = eps; run->gamma = gamma; run->dt = dt;
  run->opts = o;
  run->layout = make_layout(dim, run->n, o.coarsest);
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
    if (arena_bytes < run->layout.total || (reinterpret_cast<uintptr_t>(arena) % kAlign) != 0) {
      chhs_destroy(run);
      return CHHS_ERR_OOM;
    }
    run->arena = static_cast<char*>(arena);
  } else {
    if (cudaMalloc(&run->arena, run->layout.total) != cudaSuccess) {
      cudaGetLastError();
      run->arena = nullptr;
      chhs_destroy(run);
      return CHHS_ERR_OOM;
    }
    run->own_arena = true;
  }
  s = setup_handle(run);
  if (s != CHHS_OK) {
    chhs_destroy(run);
    return s;
  }
  *out = run;
  return CHHS_OK;
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
  return CHHS_OK;
}

size_t chhs_workspace_bytes(int dim, const int n[3], const chhs_opts* opts) {
  chhs_opts o;
  chhs_default_opts(&o);
  if (opts) o = *opts;
  if (!valid_problem(dim, n, 1.0, 1.0, 0.0, 1.0) || !valid_opts(o)) return 0;
  int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  return make_layout(dim, nn, o.coarsest).total;
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
  if (nsteps < 0) return fail(run, CHHS_ERR_INVALID_ARG, "nsteps < 0");
  run->err.clear();
  k_reset_call<<<1, 1, 0, run->stream>>>(run->st, run->opts.tol, run->opts.max_v);
  CU(cudaGetLastError());
  for (int k = 0; k < nsteps; ++k) CU(cudaGraphLaunch(run->exec, run->stream));
  return CHHS_OK;
}

chhs_status chhs_wait(chhs_t* run, int* vcycles_out, double* resid_out) {
  if (!run) return CHHS_ERR_INVALID_ARG;
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

chhs_status chhs_profile_step(chhs_t* run, double* ms_out, long long* launches_out, double* units_out) {
  if (!run || !ms_out || !launches_out || !units_out) return fail(run, CHHS_ERR_INVALID_ARG, "NULL argument");
  run->err.clear();
  Prof prof;
  run->prof = &prof;
  k_reset_call<<<1, 1, 0, run->stream>>>(run->st, run->opts.tol, run->opts.max_v);
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
  if (!run) return;
  if (run->stream) cudaStreamSynchronize(run->stream);
  if (run->exec) cudaGraphExecDestroy(run->exec);
  if (run->graph) cudaGraphDestroy(run->graph);
  if (run->host_st) cudaFreeHost(run->host_st);
  if (run->own_arena && run->arena) cudaFree(run->arena);
  if (run->own_stream && run->stream) cudaStreamDestroy(run->stream);
  delete run;
}

const char* chhs_last_error(const chhs_t* run) { return run ? run->err.c_str() : "NULL handle"; }

}  // extern "C"
