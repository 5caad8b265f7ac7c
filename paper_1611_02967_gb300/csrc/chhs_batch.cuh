// chhs_batch.cuh -- batched launches of the mixed-precision step kernels:
// one launch runs one kernel for many independent runs of uneven size.
//
// Every batched kernel takes a table of jobs (one per run that takes part:
// the arguments the run's own launch would get) and a prefix sum of the
// jobs' block counts; block b of the launch serves job j with
// start[j] <= b < start[j+1] as its block b - start[j].  The work of a block
// is the same device function, with the same arguments and block index, as
// in the run's own graph, so a run computes bit for bit what it computes
// alone.  A job whose run has stopped iterating (converged, or failed) is
// skipped by its blocks (gate: one of the run's loop flags -- go for the
// V-cycle that ends an iteration, go_more[] for the extra V-cycles a run
// takes before it when its norm predicted them, DevState::inner).
#pragma once
#include "chhs_corr3.cuh"
#include "chhs_kernels.cuh"
#include "chhs_norm_df.cuh"
#include "chhs_tile.cuh"

namespace chhs_dev {

// The job of block b: the last j with start[j] <= b (jobs without blocks
// share their start with the next job and are never chosen).
__device__ __forceinline__ int job_of(const int* start, int njobs, int b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The block's job copied into shared memory by all its threads: the device
// functions then read each field where they use it (a table in global
// memory would have its fields held in registers across the whole kernel).
template <class J>
__device__ __forceinline__ const J& job_in_smem(const J* jobs, int j) {
  __shared__ __align__(16) unsigned char buf[sizeof(J)];
  static_assert(sizeof(J) % 4 == 0, "jobs are copied as 32-bit words");
  const unsigned* src = reinterpret_cast<const unsigned*>(jobs + j);
  unsigned* dst = reinterpret_cast<unsigned*>(buf);
  for (int q = threadIdx.x; q < (int)(sizeof(J) / 4); q += blockDim.x) dst[q] = __ldg(src + q);
  __syncthreads();
  return *reinterpret_cast<const J*>(buf);
}

// A run still iterating in the V-cycle loop (its norm kernel set the flag).
__device__ __forceinline__ bool gate_open(const int* gate) {
  return gate == nullptr || *(volatile const int*)gate != 0;
}

struct SetupJob {
  Level<double> L, Cn;
  const double* phimm1;
  double eps2;
  const DevState* st;
  Coefs<double> K;
  int has_next;
};

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_setup_coef(const SetupJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const SetupJob& J = jobs[j];
  setup_coef_body<DIM>(blockIdx.x - start[j], J.L, J.phimm1, J.eps2, J.st, J.K, J.Cn, J.has_next);
}

struct CoefF32Job {
  Level<double> F;
  Level<float> G, Gn;
  Coefs<float> K;
  int has_next;
};

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_coef_restrict_f32(const CoefF32Job* jobs, const int* start,
                                                               int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const CoefF32Job& J = jobs[j];
  coef_restrict_f32_body<DIM>(blockIdx.x - start[j], J.F, J.G, J.K, J.Gn, J.has_next);
}

struct CoefJob {
  Level<float> L, Cn;
  Coefs<float> K;
  int has_next;
};

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_coef_restrict(const CoefJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const CoefJob& J = jobs[j];
  coef_restrict_body<float, DIM>(blockIdx.x - start[j], J.L, J.K, J.Cn, J.has_next);
}

struct NormJob {
  Level<double> L;
  Level<float> G;
  Coefs<double> K;
  DfCoefs Kdf;
  double* partials;
  DevState* st;
  int f64_per8;
};

// The end of a batched norm launch: every run reports once -- from its last
// block after that block has taken the run's loop decision, or from its
// block 0 when the run is not iterating and its blocks skipped the norm --
// and the launch's last report sets the loop condition to "any run still
// iterating" (also written to any_out for the host-driven profiling path).
// One atomic per run rather than per block: a launch over hundreds of runs
// has hundreds of thousands of blocks.
// any_out[0]: some run iterating; any_out[1 + q]: some run taking a
// (2 + q)-th V-cycle in its next iteration.  cc (device memory, written once
// the step graph is built; null outside the graph): the loop's condition and
// the nif IF nodes of those V-cycles.
struct BatchConds {
  cudaGraphConditionalHandle loop;
  cudaGraphConditionalHandle cif[kMaxInner - 1];
  int nif;
};

__device__ __forceinline__ void batch_norm_epilogue(const NormJob* jobs, int njobs, bool reports,
                                                    unsigned int* ticket, const BatchConds* cc,
                                                    unsigned int* any_out) {
  __shared__ bool last_run;
  __shared__ int any_go[kMaxInner];
  if (threadIdx.x == 0) {
    last_run = false;
    for (int q = 0; q < kMaxInner; ++q) any_go[q] = 0;
    if (reports) {
      __threadfence();
      last_run = atomicAdd(ticket, 1u) == (unsigned)njobs - 1;
    }
  }
  __syncthreads();
  if (!last_run) return;
  __threadfence();
  int go[kMaxInner] = {};
  for (int q = threadIdx.x; q < njobs; q += blockDim.x) {
    go[0] |= __ldcg(&jobs[q].st->go);
    for (int m = 1; m < kMaxInner; ++m) go[m] |= __ldcg(&jobs[q].st->go_more[m - 1]);
  }
  for (int m = 0; m < kMaxInner; ++m)
    if (go[m]) any_go[m] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    *ticket = 0u;
    for (int q = 0; q < kMaxInner; ++q) any_out[q] = any_go[q] ? 1u : 0u;
    if (cc) {
      cudaGraphSetConditional(cc->loop, any_go[0] ? 1u : 0u);
      for (int q = 0; q < cc->nif; ++q) cudaGraphSetConditional(cc->cif[q], any_go[1 + q] ? 1u : 0u);
    }
  }
}

// The stopping norms of all runs (mode 0: start of a step, every run; mode 1:
// after a V-cycle, the runs still iterating).  Each run's last block takes
// that run's decision.
template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_norm_mixed(const NormJob* jobs, const int* start, int njobs,
                                                        unsigned int* ticket, const BatchConds* cc, int mode,
                                                        unsigned int* any_out) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const NormJob& J = job_in_smem(jobs, j);
  const int lb = blockIdx.x - start[j];
  bool reports = lb == 0;
  if (mode == 0 || gate_open(&J.st->go))
    reports = norm_mixed_body<DIM>(lb, start[j + 1] - start[j], J.L, J.K, J.G, J.partials, J.st, 0, mode, 0);
  batch_norm_epilogue(jobs, njobs, reports, ticket, cc, any_out);
}

// The same with the double-single residual (chhs_norm_df.cuh).
template <int DIM>
__global__ void __launch_bounds__(kNdfTX * kNdfTY) kb_norm_mixed_df(const NormJob* jobs, const int* start, int njobs,
                                                                  unsigned int* ticket, const BatchConds* cc,
                                                                  int mode, unsigned int* any_out) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const NormJob& J = job_in_smem(jobs, j);
  const int lb = blockIdx.x - start[j];
  bool reports = lb == 0;
  if (mode == 0 || gate_open(&J.st->go))
    reports = norm_mixed_df_body<DIM>(lb, start[j + 1] - start[j], J.L, J.Kdf, J.K, J.f64_per8, J.G, J.partials,
                                      J.st, 0, mode, 0);
  batch_norm_epilogue(jobs, njobs, reports, ticket, cc, any_out);
}

template <typename T>
struct TileJob {
  Level<T> L, C;
  Coefs<T> K;
  TileOut<T> out;
  const int* gate;
  int npass, halo, rhs, prolong, restrict_out;
  int gx;  // tiles per row of the level
};

template <typename T, bool CORR>
__global__ void __launch_bounds__(kTileThreads, 3) kb_tile(const TileJob<T>* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const TileJob<T>& J = job_in_smem(jobs, j);
  if (!gate_open(J.gate)) return;
  const int lb = blockIdx.x - start[j];
  const int by = lb / J.gx, bx = lb - by * J.gx;
  tile_body<T, CORR>(bx, by, J.L, J.C, J.K, J.npass, J.halo, J.rhs, J.prolong, J.restrict_out, J.out);
}

template <typename T>
struct TailJob {
  Tail<T> tl;
  Coefs<T> K;
  const int* gate;
};

// One block per job.
template <typename T, int DIM, bool CORR>
__global__ void __launch_bounds__(kTailThreads, 1) kb_tail(const TailJob<T>* jobs) {
  pdl_enter();
  const TailJob<T>& J = jobs[blockIdx.x];
  if (!gate_open(J.gate)) return;
  tail_body<T, DIM, CORR>(J.tl, J.K);
}

struct SmoothCJob {
  Level<float> L, C;
  Level<double> U;
  Coefs<float> K;
  const int* gate;
  int colour, rhs, pro;
};

template <int DIM>
__global__ void __launch_bounds__(kSmoothBlock) kb_smooth_c(const SmoothCJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const SmoothCJob& J = job_in_smem(jobs, j);
  if (!gate_open(J.gate)) return;
  smooth_c_body<DIM>(blockIdx.x - start[j], J.L, J.C, J.K, J.colour, J.rhs, J.pro, J.U);
}

// Two-level jobs (residual-restriction, prolongation, coarse right-hand side)
// and the double-precision update.
struct PairJob {
  Level<float> F, C;
  Coefs<float> K;
  Level<double> U;
  const int* gate;
};

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_residual_restrict_c(const PairJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const PairJob& J = job_in_smem(jobs, j);
  if (!gate_open(J.gate)) return;
  residual_restrict_c_body<DIM>(blockIdx.x - start[j], J.F, J.C, J.K);
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_prolong(const PairJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const PairJob& J = jobs[j];
  if (!gate_open(J.gate)) return;
  prolong_body<float, DIM>(blockIdx.x - start[j], J.F, J.C);
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) kb_coarse_rhs(const PairJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const PairJob& J = jobs[j];
  if (!gate_open(J.gate)) return;
  coarse_rhs_body<float, DIM, true>(blockIdx.x - start[j], J.F, J.K);
}

static __global__ void __launch_bounds__(kBlock) kb_mixed_update(const PairJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const PairJob& J = jobs[j];
  if (!gate_open(J.gate)) return;
  mixed_update_body(blockIdx.x - start[j], J.U, J.F);
}

struct AdvanceJob {
  Level<double> L;
  double* phimm1;
  DevState* st;
};

static __global__ void __launch_bounds__(kBlock) kb_advance(const AdvanceJob* jobs, const int* start, int njobs) {
  pdl_enter();
  const int j = job_of(start, njobs, blockIdx.x);
  const AdvanceJob& J = jobs[j];
  advance_body(blockIdx.x - start[j], J.L, J.phimm1, J.st);
}

// The start of a batched call: every run's counters reset (one thread per run).
static __global__ void kb_reset(DevState* const* sts, int nruns, double tol, double tol_max, int max_v,
                                int max_inner) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  DevState* st = sts[r];
  st->failed = 0;
  st->vtotal = 0;
  st->steps_done = 0;
  st->checks = 0;
  st->tol = tol;
  st->tol_max = tol_max;
  st->max_v = max_v;
  st->max_inner = max_inner;
}

// Every run's outcome of a call: status, V-cycles (as chhs_wait reports
// them) and the last stopping norm, gathered for one copy to the host.
static __global__ void kb_gather(DevState* const* sts, int nruns, int* status, int* vcycles, double* resid) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  const DevState* st = sts[r];
  status[r] = st->failed;
  vcycles[r] = st->vtotal + (st->failed ? st->vcycles : 0);
  resid[r] = st->resid;
}

}  // namespace chhs_dev
