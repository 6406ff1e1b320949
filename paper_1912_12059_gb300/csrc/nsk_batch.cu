// nsk_batch.cu -- batched execution of many 3D contexts (meshes of different sizes,
// N = 3 or 4) in one persistent launch per LSRK stage.
//
// The four stage phases (trace prolongation, BR1 lifting, face fluxes, volume
// integral + update) of every instance run inside one cooperative kernel (with the
// separate face schedule the volume phase writes the next stage's traces, so a
// step's stages skip the prolongation: one prolongation pass per nsk_batch_step),
// separated by a grid barrier whose spin is bounded in time: on expiry the
// kernel sets NSK_EBIT_TIMEOUT and returns instead of waiting forever. Work
// units (trace items, element groups, face items) of all instances are
// concatenated and striped over the grid, so small instances fill the GPU
// together. The five stage launches of a step (and, optionally, the per-
// instance time-step reductions) are captured once in a CUDA graph and the
// graph is replayed per step. An autotuner times the block-size and face
// schedules, and the instance schedule (each instance's own stage launches in
// the graph, for instances that fill the GPU alone), and keeps the fastest.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "nsk_kernels.cuh"
#include "nsk_nvtx.h"
#include "nsk_test_hooks.h"

// Device descriptor of one instance.
struct BatchInst {
  NskParams p;
  void *U, *K, *Q, *Utr, *FVtr, *Fstar, *Rout;
  const double* dt;
  long long off[4];  // first global work unit of this instance in each phase
  long long cnt[4];  // work units: chunks of blockDim trace items, element groups, chunks of face items, groups
  long long items[4];  // trace items and face items (phases 0 and 2)
  int np;
};

struct nsk_batch {
  int n, precision, tpb, fused, persistent;
  std::vector<nsk_ctx*> inst;
  BatchInst* d_inst;
  unsigned* d_bar;  // grid barrier: [0] arrivals, [1] generation
  int* d_err;
  cudaStream_t stream;
  long long tot[2][2][4];  // [tpb index][fused][phase]
  std::vector<BatchInst> h_inst[2];  // per tpb choice
  cudaGraphExec_t graph;
  int graph_tpb, graph_fused, graph_dtmode, graph_persistent;
  unsigned long long graph_inst_sched;  // the instances' own schedules the graph was captured with
  double graph_cfl;
  bool no_graph;          // capture or instantiation unavailable: stages launched directly
  long long launches;
  long long graph_launches;  // kernel launches of the captured stages of one step
  // per-phase schedule: its own work-unit offsets (item phases in chunks of TPB * items per
  // thread) and block -> instance maps
  BatchInst* d_pinst;
  long long ptot[2][4];
  int* d_blk2inst[2][4];
  int grid[2][2];         // co-resident grid size per [tpb index][fused]
  unsigned long long timeout_ns;  // bound of every grid-barrier wait
  // per-instance step latency (nsk_batch_step with per_instance_latency_ms): global-timer stamps
  // [0] step start, [1 + i] step done for instance i, written by tiny kernels inside the step's
  // graph; after every step they are copied into a history of steps read back at the end
  unsigned long long* d_stamp;
  unsigned long long* d_hist;
  long long hist_cap;      // steps the history holds
  int graph_stamps;        // the captured graph carries the stamp kernels
  // instance schedule: instance i launches on aux[i % naux], forked from and joined back to stream
  // around every stage (small instances that cannot fill the GPU alone run side by side)
  static constexpr int kAux = 4;
  int naux;
  cudaStream_t aux[kAux];
  cudaEvent_t ev_fork, ev_join[kAux];
};

namespace {

using nsk::grid_barrier;

constexpr int align16(int x) { return (x + 15) & ~15; }

template <typename R, int TPB, bool FUSED>
constexpr int batch_smem_bytes() {
  constexpr int G4 = nsk::group_for<3, 4>(TPB), G5 = nsk::group_for<3, 5>(TPB);
  constexpr int a = nsk::lift_smem<R, 3, 4, G4>(), b = nsk::lift_smem<R, 3, 5, G5>();
  constexpr int c = nsk::volume_smem<R, 3, 4, G4, FUSED>(), d = nsk::volume_smem<R, 3, 5, G5, FUSED>();
  constexpr int m1 = a > b ? a : b, m2 = c > d ? c : d;
  return align16((int)sizeof(NskParams)) + (int)sizeof(R) * (m1 > m2 ? m1 : m2);
}

// copy an instance's parameters into shared memory (all threads of the block)
__device__ __forceinline__ void load_params(NskParams* sp, const NskParams* gp) {
  const int nw = (int)(sizeof(NskParams) / sizeof(int));
  const int* src = (const int*)gp;
  int* dst = (int*)sp;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
}

// occupancy target of the persistent kernel: it carries every phase's registers at once,
// so the bound keeps 32 (FP32) or 24 (FP64) warps per SM resident
template <typename R, int TPB>
constexpr int batch_min_blocks() {
  return (sizeof(R) == 4 ? 1024 : 768) / TPB;
}

template <typename R, int TPB, bool FUSED>
__global__ void __launch_bounds__(TPB, batch_min_blocks<R, TPB>())
    k_batch_stage(const BatchInst* __restrict__ inst, const int ninst, const long long tot0, const long long tot1,
                  const long long tot2, const long long tot3, const int mode, const R A, const R B,
                  unsigned* __restrict__ bar, int* __restrict__ err, const unsigned long long timeout_ns,
                  const int traces) {
  constexpr int G4 = nsk::group_for<3, 4>(TPB), G5 = nsk::group_for<3, 5>(TPB);
  extern __shared__ __align__(16) unsigned char smraw[];
  NskParams* sp = (NskParams*)smraw;
  R* sm = (R*)(smraw + align16((int)sizeof(NskParams)));
  int eflag = 0;

  // phase 0: traces of U on every face, one chunk of TPB items of one instance per block iteration
  // (skipped when the previous stage's volume phase already wrote them: traces bit 0)
  if (!(traces & 1)) {
    int i = 0, cur = -1;
    for (long long ci = blockIdx.x; ci < tot0; ci += gridDim.x) {
      while (ci >= inst[i].off[0] + inst[i].cnt[0]) ++i;
      if (i != cur) {
        __syncthreads();
        load_params(sp, &inst[i].p);
        __syncthreads();
        cur = i;
      }
      const BatchInst& b = inst[i];
      const long long it = (ci - b.off[0]) * TPB + threadIdx.x;
      if (it < b.items[0]) {
        if (b.np == 4)
          nsk::prolong_item<R, 3, 4>(*sp, (const R*)b.U, (R*)b.Utr, it);
        else
          nsk::prolong_item<R, 3, 5>(*sp, (const R*)b.U, (R*)b.Utr, it);
      }
    }
  }
  if (!(traces & 1) && !grid_barrier(bar, err, timeout_ns)) return;

  // phase 1: BR1 lifting, one element group per block iteration
  {
    int i = 0, cur = -1;
    for (long long gi = blockIdx.x; gi < tot1; gi += gridDim.x) {
      while (gi >= inst[i].off[1] + inst[i].cnt[1]) ++i;
      if (i != cur) {
        __syncthreads();
        load_params(sp, &inst[i].p);
        __syncthreads();
        cur = i;
      }
      const BatchInst& b = inst[i];
      const long long loc = gi - b.off[1];
      if (b.np == 4)
        nsk::lift_group<R, 3, 4, G4>(*sp, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr, loc * G4, sm, eflag);
      else
        nsk::lift_group<R, 3, 5, G5>(*sp, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr, loc * G5, sm, eflag);
    }
  }
  if (!grid_barrier(bar, err, timeout_ns)) return;

  // phase 2: face fluxes (separate face schedule)
  if (!FUSED) {
    int i = 0, cur = -1;
    for (long long ci = blockIdx.x; ci < tot2; ci += gridDim.x) {
      while (ci >= inst[i].off[2] + inst[i].cnt[2]) ++i;
      if (i != cur) {
        __syncthreads();
        load_params(sp, &inst[i].p);
        __syncthreads();
        cur = i;
      }
      const BatchInst& b = inst[i];
      const long long it = (ci - b.off[2]) * TPB + threadIdx.x;
      if (it < b.items[2]) {
        if (b.np == 4)
          nsk::face_item<R, 3, 4>(*sp, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.Fstar, it, eflag);
        else
          nsk::face_item<R, 3, 5>(*sp, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.Fstar, it, eflag);
      }
    }
    if (!grid_barrier(bar, err, timeout_ns)) return;
  }

  // phase 3: volume integral, surface lifting, sources, update
  {
    int i = 0, cur = -1;
    R dt = 0;
    for (long long gi = blockIdx.x; gi < tot3; gi += gridDim.x) {
      while (gi >= inst[i].off[3] + inst[i].cnt[3]) ++i;
      if (i != cur) {
        __syncthreads();
        load_params(sp, &inst[i].p);
        __syncthreads();
        cur = i;
        dt = inst[i].dt ? (R)*inst[i].dt : R(0);
      }
      const BatchInst& b = inst[i];
      const long long loc = gi - b.off[3];
      // traces bit 1 (separate face schedule only: the volume phase then reads no traces):
      // write the traces of the updated state in place for the next stage
      R* tnext = (!FUSED && (traces & 2)) ? (R*)b.Utr : nullptr;
      if (b.np == 4)
        nsk::volume_group<R, 3, 4, G4, FUSED>(*sp, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr,
                                              (const R*)b.FVtr, (R*)b.K, (R*)b.Rout, mode, A, B, dt, loc * G4, sm,
                                              eflag, tnext);
      else
        nsk::volume_group<R, 3, 5, G5, FUSED>(*sp, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr,
                                              (const R*)b.FVtr, (R*)b.K, (R*)b.Rout, mode, A, B, dt, loc * G5, sm,
                                              eflag, tnext);
    }
  }
  if (eflag) atomicOr(err, eflag);
}

// ---- per-phase batched kernels: one launch per phase over all instances ---------
// Block b handles work unit b of the phase: the instance is found by binary search
// over the per-instance offsets (uniform in the block), its parameters staged in
// shared memory. Each phase is its own kernel, so each keeps its own register budget.
constexpr int kItemsPerThread = 4;  // item phases of the per-phase schedule: items per thread

template <typename R, int TPB>
__global__ void __launch_bounds__(TPB) k_bphase_prolong(const BatchInst* __restrict__ inst,
                                                        const int* __restrict__ blk2inst) {
  __shared__ __align__(16) unsigned char spraw[sizeof(NskParams)];
  NskParams* sp = (NskParams*)spraw;
  const int i = blk2inst[blockIdx.x];
  load_params(sp, &inst[i].p);
  __syncthreads();
  const BatchInst& b = inst[i];
  const long long base = ((long long)blockIdx.x - b.off[0]) * TPB * kItemsPerThread + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const long long it = base + (long long)r * TPB;
    if (it < b.items[0]) {
      if (b.np == 4)
        nsk::prolong_item<R, 3, 4>(*sp, (const R*)b.U, (R*)b.Utr, it);
      else
        nsk::prolong_item<R, 3, 5>(*sp, (const R*)b.U, (R*)b.Utr, it);
    }
  }
}

template <typename R, int TPB>
__global__ void __launch_bounds__(TPB, (nsk::lift_min_blocks<R, TPB>())) k_bphase_lift(const BatchInst* __restrict__ inst,
                                                     const int* __restrict__ blk2inst, int* __restrict__ err) {
  constexpr int G4 = nsk::group_for<3, 4>(TPB), G5 = nsk::group_for<3, 5>(TPB);
  constexpr int a = nsk::lift_smem<R, 3, 4, G4>(), c = nsk::lift_smem<R, 3, 5, G5>();
  __shared__ R sm[a > c ? a : c];
  __shared__ __align__(16) unsigned char spraw[sizeof(NskParams)];
  NskParams* sp = (NskParams*)spraw;
  const int i = blk2inst[blockIdx.x];
  load_params(sp, &inst[i].p);
  __syncthreads();
  const BatchInst& b = inst[i];
  const long long loc = (long long)blockIdx.x - b.off[1];
  int eflag = 0;
  if (b.np == 4)
    nsk::lift_group<R, 3, 4, G4>(*sp, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr, loc * G4, sm, eflag);
  else
    nsk::lift_group<R, 3, 5, G5>(*sp, (const R*)b.U, (const R*)b.Utr, (R*)b.Q, (R*)b.FVtr, loc * G5, sm, eflag);
  if (eflag) atomicOr(err, eflag);
}

template <typename R, int TPB>
__global__ void __launch_bounds__(TPB) k_bphase_face(const BatchInst* __restrict__ inst,
                                                     const int* __restrict__ blk2inst, int* __restrict__ err) {
  __shared__ __align__(16) unsigned char spraw[sizeof(NskParams)];
  NskParams* sp = (NskParams*)spraw;
  const int i = blk2inst[blockIdx.x];
  load_params(sp, &inst[i].p);
  __syncthreads();
  const BatchInst& b = inst[i];
  const long long base = ((long long)blockIdx.x - b.off[2]) * TPB * kItemsPerThread + threadIdx.x;
  int eflag = 0;
#pragma unroll
  for (int r = 0; r < kItemsPerThread; ++r) {
    const long long it = base + (long long)r * TPB;
    if (it < b.items[2]) {
      if (b.np == 4)
        nsk::face_item<R, 3, 4>(*sp, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.Fstar, it, eflag);
      else
        nsk::face_item<R, 3, 5>(*sp, (const R*)b.Utr, (const R*)b.FVtr, (R*)b.Fstar, it, eflag);
    }
  }
  if (eflag) atomicOr(err, eflag);
}

template <typename R, int TPB, bool FUSED>
__global__ void __launch_bounds__(TPB) k_bphase_volume(const BatchInst* __restrict__ inst,
                                                       const int* __restrict__ blk2inst, const int mode, const R A,
                                                       const R B, int* __restrict__ err, const int write_traces) {
  constexpr int G4 = nsk::group_for<3, 4>(TPB), G5 = nsk::group_for<3, 5>(TPB);
  constexpr int a = nsk::volume_smem<R, 3, 4, G4, FUSED>(), c = nsk::volume_smem<R, 3, 5, G5, FUSED>();
  __shared__ R sm[a > c ? a : c];
  __shared__ __align__(16) unsigned char spraw[sizeof(NskParams)];
  NskParams* sp = (NskParams*)spraw;
  const int i = blk2inst[blockIdx.x];
  load_params(sp, &inst[i].p);
  __syncthreads();
  const BatchInst& b = inst[i];
  const long long loc = (long long)blockIdx.x - b.off[3];
  const R dt = b.dt ? (R)*b.dt : R(0);
  R* tnext = (!FUSED && write_traces) ? (R*)b.Utr : nullptr;
  int eflag = 0;
  if (b.np == 4)
    nsk::volume_group<R, 3, 4, G4, FUSED>(*sp, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr,
                                          (const R*)b.FVtr, (R*)b.K, (R*)b.Rout, mode, A, B, dt, loc * G4, sm,
                                          eflag, tnext);
  else
    nsk::volume_group<R, 3, 5, G5, FUSED>(*sp, (R*)b.U, (const R*)b.Q, (const R*)b.Fstar, (const R*)b.Utr,
                                          (const R*)b.FVtr, (R*)b.K, (R*)b.Rout, mode, A, B, dt, loc * G5, sm,
                                          eflag, tnext);
  if (eflag) atomicOr(err, eflag);
}

const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};

// shared-memory attribute and co-resident grid size of one variant (outside any capture)
template <typename R, int TPB, bool FUSED>
int prepare_batch_t(nsk_batch* bt) {
  auto kern = k_batch_stage<R, TPB, FUSED>;
  constexpr int smem = batch_smem_bytes<R, TPB, FUSED>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return NSK_ERR_CUDA;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, smem) != cudaSuccess || per_sm < 1)
    return NSK_ERR_CUDA;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NSK_ERR_CUDA;
  const int ti = TPB == 128 ? 0 : 1;
  const long long* tot = bt->tot[ti][FUSED ? 1 : 0];
  long long want = tot[0];
  for (int ph = 1; ph < 4; ++ph) want = tot[ph] > want ? tot[ph] : want;
  long long grid = (long long)per_sm * sms;
  if (want < grid) grid = want > 0 ? want : 1;
  bt->grid[ti][FUSED ? 1 : 0] = (int)grid;
  return NSK_OK;
}

template <typename R, int TPB, bool FUSED>
int launch_batch_t(nsk_batch* bt, int mode, double A, double B, int traces) {
  auto kern = k_batch_stage<R, TPB, FUSED>;
  constexpr int smem = batch_smem_bytes<R, TPB, FUSED>();
  const int ti = TPB == 128 ? 0 : 1;
  const long long* tot = bt->tot[ti][FUSED ? 1 : 0];
  const int grid = bt->grid[ti][FUSED ? 1 : 0];
  if (grid < 1) return NSK_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TPB);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = bt->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BatchInst* d_inst = bt->d_inst + (size_t)ti * bt->n;
  if (cudaLaunchKernelEx(&cfg, kern, d_inst, bt->n, tot[0], tot[1], tot[2], tot[3], mode, (R)A, (R)B, bt->d_bar,
                         bt->d_err, bt->timeout_ns, traces) != cudaSuccess)
    return NSK_ERR_CUDA;
  bt->launches += 1;
  return NSK_OK;
}

// traces: bit 0 = the face traces of U are current (no prolongation phase), bit 1 = the volume
// phase writes the traces of its output state (separate face schedule only)
template <typename R, int TPB, bool FUSED>
int launch_phases_t(nsk_batch* bt, int mode, double A, double B, int traces) {
  const int ti = TPB == 128 ? 0 : 1;
  const long long* tot = bt->ptot[ti];
  const BatchInst* d_inst = bt->d_pinst + (size_t)ti * bt->n;
  const int* const* map = bt->d_blk2inst[ti];
  cudaStream_t s = bt->stream;
  int nl = 0;
  if (!(traces & 1)) {
    k_bphase_prolong<R, TPB><<<(unsigned)tot[0], TPB, 0, s>>>(d_inst, map[0]);
    ++nl;
  }
  k_bphase_lift<R, TPB><<<(unsigned)tot[1], TPB, 0, s>>>(d_inst, map[1], bt->d_err);
  ++nl;
  if (!FUSED) {
    k_bphase_face<R, TPB><<<(unsigned)tot[2], TPB, 0, s>>>(d_inst, map[2], bt->d_err);
    ++nl;
  }
  k_bphase_volume<R, TPB, FUSED><<<(unsigned)tot[3], TPB, 0, s>>>(d_inst, map[3], mode, (R)A, (R)B, bt->d_err,
                                                                  (traces >> 1) & 1);
  ++nl;
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  bt->launches += nl;
  return NSK_OK;
}

// the prolongation phase alone (per-phase kernel), for all instances
template <typename R, int TPB>
int launch_prolong_t(nsk_batch* bt) {
  const int ti = TPB == 128 ? 0 : 1;
  k_bphase_prolong<R, TPB><<<(unsigned)bt->ptot[ti][0], TPB, 0, bt->stream>>>(bt->d_pinst + (size_t)ti * bt->n,
                                                                               bt->d_blk2inst[ti][0]);
  if (cudaGetLastError() != cudaSuccess) return NSK_ERR_CUDA;
  bt->launches += 1;
  return NSK_OK;
}

int launch_prolong(nsk_batch* bt, int tpb) {
  const bool f32 = bt->precision == NSK_FP32_MIXED;
  if (tpb == 128) return f32 ? launch_prolong_t<float, 128>(bt) : launch_prolong_t<double, 128>(bt);
  return f32 ? launch_prolong_t<float, 256>(bt) : launch_prolong_t<double, 256>(bt);
}

int launch_phases(nsk_batch* bt, int mode, double A, double B, int tpb, int fused, int tr) {
  const bool f32 = bt->precision == NSK_FP32_MIXED;
  if (tpb == 128) {
    if (f32) return fused ? launch_phases_t<float, 128, true>(bt, mode, A, B, tr) : launch_phases_t<float, 128, false>(bt, mode, A, B, tr);
    return fused ? launch_phases_t<double, 128, true>(bt, mode, A, B, tr) : launch_phases_t<double, 128, false>(bt, mode, A, B, tr);
  }
  if (f32) return fused ? launch_phases_t<float, 256, true>(bt, mode, A, B, tr) : launch_phases_t<float, 256, false>(bt, mode, A, B, tr);
  return fused ? launch_phases_t<double, 256, true>(bt, mode, A, B, tr) : launch_phases_t<double, 256, false>(bt, mode, A, B, tr);
}

int launch_persistent(nsk_batch* bt, int mode, double A, double B, int tpb, int fused, int tr) {
  const bool f32 = bt->precision == NSK_FP32_MIXED;
  if (tpb == 128) {
    if (f32) return fused ? launch_batch_t<float, 128, true>(bt, mode, A, B, tr) : launch_batch_t<float, 128, false>(bt, mode, A, B, tr);
    return fused ? launch_batch_t<double, 128, true>(bt, mode, A, B, tr) : launch_batch_t<double, 128, false>(bt, mode, A, B, tr);
  }
  if (f32) return fused ? launch_batch_t<float, 256, true>(bt, mode, A, B, tr) : launch_batch_t<float, 256, false>(bt, mode, A, B, tr);
  return fused ? launch_batch_t<double, 256, true>(bt, mode, A, B, tr) : launch_batch_t<double, 256, false>(bt, mode, A, B, tr);
}

int prepare_batch(nsk_batch* bt) {
  int st;
  if (bt->precision == NSK_FP32_MIXED) {
    if ((st = prepare_batch_t<float, 128, false>(bt)) || (st = prepare_batch_t<float, 128, true>(bt)) ||
        (st = prepare_batch_t<float, 256, false>(bt)) || (st = prepare_batch_t<float, 256, true>(bt)))
      return st;
  } else {
    if ((st = prepare_batch_t<double, 128, false>(bt)) || (st = prepare_batch_t<double, 128, true>(bt)) ||
        (st = prepare_batch_t<double, 256, false>(bt)) || (st = prepare_batch_t<double, 256, true>(bt)))
      return st;
  }
  return NSK_OK;
}

// slot[i] = the global timer (ns), i < n: the step-start stamp (n = 1) or the completion stamp
// of instances whose work ended with the previous launch on the stream (stream order)
__global__ void k_stamp(unsigned long long* __restrict__ slot, const int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) slot[i] = nsk::global_ns();
}

int launch_stamp(nsk_batch* bt, unsigned long long* slot, int n, cudaStream_t s = nullptr) {
  k_stamp<<<(n + 255) / 256, 256, 0, s ? s : bt->stream>>>(slot, n);
  ++bt->launches;
  return cudaGetLastError() == cudaSuccess ? NSK_OK : NSK_ERR_CUDA;
}

// the instance schedule's streams: fork from the batch stream before a stage, join after it
int fork_aux(nsk_batch* bt) {
  if (bt->naux < 2) return NSK_OK;
  if (cudaEventRecord(bt->ev_fork, bt->stream) != cudaSuccess) return NSK_ERR_CUDA;
  for (int j = 0; j < bt->naux; ++j)
    if (cudaStreamWaitEvent(bt->aux[j], bt->ev_fork, 0) != cudaSuccess) return NSK_ERR_CUDA;
  return NSK_OK;
}
int join_aux(nsk_batch* bt) {
  if (bt->naux < 2) return NSK_OK;
  for (int j = 0; j < bt->naux; ++j)
    if (cudaEventRecord(bt->ev_join[j], bt->aux[j]) != cudaSuccess ||
        cudaStreamWaitEvent(bt->stream, bt->ev_join[j], 0) != cudaSuccess)
      return NSK_ERR_CUDA;
  return NSK_OK;
}
cudaStream_t inst_stream(const nsk_batch* bt, int i) { return bt->naux < 2 ? bt->stream : bt->aux[i % bt->naux]; }

// instance schedule: every instance's own stage kernels, instance i on stream i mod naux; with
// stamps (the last stage of a step whose latencies are measured) each instance's completion
// is stamped right after its last kernel
// fused 5: each instance's own schedule (its tpb and fused_face; the lean and single-block schedules
// run as the separate face pass there)
int inst_fused(const nsk_ctx* c) { return (c->fused_face == 1 || c->fused_face == 4) ? c->fused_face : 0; }
int launch_instances(nsk_batch* bt, int mode, double A, double B, int tpb, int fused, int traces,
                     bool stamps = false) {
  for (int i = 0; i < bt->n; ++i) {
    nsk_ctx* c = bt->inst[i];
    const int fi = fused == 5 ? inst_fused(c) : fused;
    const int tr = fi == 1 ? 0 : traces;  // the fused volume phase prolongs every stage
    NskLaunch l = {mode, c->rbuf, A, B, c->b.dt, 0.0, nullptr, fused == 5 ? c->tpb : tpb, fi};
    l.traces_ready = tr & 1;
    l.utr_next = (tr & 2) ? c->b.Utr : nullptr;  // separate face schedule: written in place
    const int r = nsk_launch_stage_d3(c->p, c->np, c->precision == NSK_FP32_MIXED, c->b, l, inst_stream(bt, i));
    if (r < 0) return r;
    bt->launches += r;
    if (stamps) {
      const int st = launch_stamp(bt, bt->d_stamp + 1 + i, 1, inst_stream(bt, i));
      if (st) return st;
    }
  }
  return NSK_OK;
}

// the lean stage on every instance (instance schedule, fused_face 2): a step prolongs once into
// each instance's trace buffer (stage 0), then its stages alternate between that buffer and the
// instance's spare one (the lean volume kernel writes the next stage's traces while its
// neighbours still read the current ones); the last stage of a step writes none. stage < 0: a
// residual (prolongation, no traces written).
int launch_instances_lean(nsk_batch* bt, int mode, double A, double B, int tpb, int stage, bool stamps) {
  for (int i = 0; i < bt->n; ++i) {
    nsk_ctx* c = bt->inst[i];
    NskBuffers b = c->b;
    void* bufs[2] = {c->b.Utr, c->utr_alt};
    NskLaunch l = {mode, c->rbuf, A, B, c->b.dt, 0.0, nullptr, tpb, 2};
    if (stage >= 0) {
      b.Utr = bufs[stage & 1];
      l.traces_ready = stage > 0;
      l.utr_next = stage < 4 ? bufs[(stage + 1) & 1] : nullptr;
    }
    const int r = nsk_launch_stage_d3(c->p, c->np, c->precision == NSK_FP32_MIXED, b, l, inst_stream(bt, i));
    if (r < 0) return r;
    bt->launches += r;
    if (stamps) {
      const int st = launch_stamp(bt, bt->d_stamp + 1 + i, 1, inst_stream(bt, i));
      if (st) return st;
    }
  }
  return NSK_OK;
}

// the instances' schedules as one number (tpb and effective fused_face of each, in order)
unsigned long long inst_schedules(const nsk_batch* bt) {
  unsigned long long h = 1469598103934665603ull;  // FNV-1a over the pairs
  for (const nsk_ctx* c : bt->inst) {
    h = (h ^ (unsigned long long)(c->tpb == 128 ? 1 : 2)) * 1099511628211ull;
    h = (h ^ (unsigned long long)inst_fused(c)) * 1099511628211ull;
  }
  return h;
}

// one stage of the whole batch under a schedule (persistent 1: one cooperative launch; 0: one
// launch per phase; 2: every instance's own launches)
// trace flags of every stage of a step under the separate face schedule: traces come from the
// previous stage's volume phase (the step starts from traces prolonged before the first step)
// (the line schedule, fused_face 4, is a separate face schedule)
int step_traces(int fused) { return (fused == 0 || fused == 4 || fused == 5) ? 3 : 0; }

// stamps: the last stage of a step whose per-instance latencies are measured (each instance's
// completion stamped after its last kernel; one launch for all instances stamps them together)
int launch_batch(nsk_batch* bt, int mode, double A, double B, int tpb, int fused, int persistent, int traces,
                 bool stamps = false, int stage = -1) {
  if (persistent == 2) {  // the instance schedule, forked onto the auxiliary streams
    int r = fork_aux(bt);
    if (r) return r;
    if (fused == 2)
      r = launch_instances_lean(bt, mode, A, B, tpb, stage, stamps);
    else
      r = launch_instances(bt, mode, A, B, tpb, fused, fused == 1 ? 0 : traces, stamps);
    const int j = join_aux(bt);
    return r ? r : j;
  }
  if (fused == 1) traces = 0;  // the fused volume phase reads the traces: they are prolonged every stage
  const int r = persistent ? launch_persistent(bt, mode, A, B, tpb, fused, traces)
                           : launch_phases(bt, mode, A, B, tpb, fused, traces);
  if (r || !stamps) return r;
  return launch_stamp(bt, bt->d_stamp + 1, bt->n);
}

// the launches of one step: per-instance dt reductions (cfl > 0), then the five stages; with
// stamps the step start and every instance's completion are stamped
int launch_step(nsk_batch* bt, int dtmode, double cfl, bool stamps) {
  if (stamps) {
    const int st = launch_stamp(bt, bt->d_stamp, 1);
    if (st) return st;
  }
  if (dtmode)
    for (nsk_ctx* c : bt->inst) {
      const int r = nsk_launch_dt(c->p, c->dim, c->np, c->precision == NSK_FP32_MIXED, c->b, cfl, bt->stream);
      if (r < 0) return r;
      bt->launches += r;
    }
  for (int s = 0; s < 5; ++s) {
    const int r = launch_batch(bt, NSK_MODE_LSRK, kA[s], kB[s], bt->tpb, bt->fused, bt->persistent,
                               step_traces(bt->fused), stamps && s == 4, s);
    if (r) return r;
  }
  return NSK_OK;
}


int read_error(nsk_batch* bt) {
  int h = 0;
  if (cudaMemcpyAsync(&h, bt->d_err, sizeof(int), cudaMemcpyDeviceToHost, bt->stream) != cudaSuccess ||
      cudaStreamSynchronize(bt->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  if (h) {
    // clear the error word and the barrier (a timed-out barrier leaves arrivals behind)
    cudaMemsetAsync(bt->d_err, 0, sizeof(int), bt->stream);
    cudaMemsetAsync(bt->d_bar, 0, 2 * sizeof(unsigned), bt->stream);
    cudaStreamSynchronize(bt->stream);
    return (h & NSK_EBIT_TIMEOUT) ? NSK_ERR_TIMEOUT : NSK_ERR_NONPHYSICAL;
  }
  return NSK_OK;
}

void destroy_graph(nsk_batch* bt) {
  if (bt->graph) cudaGraphExecDestroy(bt->graph);
  bt->graph = nullptr;
}

}  // namespace

extern "C" {

int nsk_batch_create(nsk_batch** out, int n, nsk_ctx* const* instances) {
  if (!out || n < 1 || !instances) return NSK_ERR_ARG;
  *out = nullptr;
  const int prec = instances[0] ? instances[0]->precision : -1;
  for (int i = 0; i < n; ++i) {
    nsk_ctx* c = instances[i];
    if (!c || c->dim != 3 || (c->np != 4 && c->np != 5) || c->precision != prec || c->p.model != NSK_MODEL_RELAXATION)
      return NSK_ERR_ARG;
    if (!c->state_set) return NSK_ERR_STATE;
  }
  nsk_batch* bt = new (std::nothrow) nsk_batch();
  if (!bt) return NSK_ERR_NOMEM;
  bt->n = n;
  bt->precision = prec;
  bt->tpb = 256;
  bt->fused = 0;
  bt->persistent = 1;
  bt->timeout_ns = 1000000000ull;  // one second per barrier wait
  bt->inst.assign(instances, instances + n);
  const int tpbs[2] = {128, 256};
  for (int ti = 0; ti < 2; ++ti) {
    bt->h_inst[ti].resize(n);
    for (int f = 0; f < 2; ++f)
      for (int ph = 0; ph < 4; ++ph) bt->tot[ti][f][ph] = 0;
    for (int i = 0; i < n; ++i) {
      nsk_ctx* c = instances[i];
      BatchInst& b = bt->h_inst[ti][i];
      memset(&b, 0, sizeof(b));
      b.p = c->p;
      b.U = c->b.U;
      b.K = c->b.K;
      b.Q = c->b.Q;
      b.Utr = c->b.Utr;
      b.FVtr = c->b.FVtr;
      b.Fstar = c->b.Fstar;
      b.Rout = c->rbuf;
      b.dt = c->b.dt;
      b.np = c->np;
      const int G = c->np == 4 ? (tpbs[ti] / 64 > 0 ? tpbs[ti] / 64 : 1) : (tpbs[ti] / 125 > 0 ? tpbs[ti] / 125 : 1);
      b.items[0] = c->E * 6 * c->nfn;
      b.items[2] = c->E * 3 * c->nfn;
      b.cnt[0] = (b.items[0] + tpbs[ti] - 1) / tpbs[ti];
      b.cnt[1] = (c->E + G - 1) / G;
      b.cnt[2] = (b.items[2] + tpbs[ti] - 1) / tpbs[ti];
      b.cnt[3] = b.cnt[1];
      for (int ph = 0; ph < 4; ++ph) {
        b.off[ph] = bt->tot[ti][0][ph];
        bt->tot[ti][0][ph] += b.cnt[ph];
      }
    }
    for (int ph = 0; ph < 4; ++ph) bt->tot[ti][1][ph] = bt->tot[ti][0][ph];
  }
  std::vector<BatchInst> pinst[2];
  std::vector<int> maps[2][4];
  for (int ti = 0; ti < 2; ++ti) {
    pinst[ti] = bt->h_inst[ti];
    for (int ph = 0; ph < 4; ++ph) bt->ptot[ti][ph] = 0;
    for (int i = 0; i < n; ++i) {
      BatchInst& b = pinst[ti][i];
      const long long chunk = (long long)tpbs[ti] * kItemsPerThread;
      b.cnt[0] = (b.items[0] + chunk - 1) / chunk;
      b.cnt[2] = (b.items[2] + chunk - 1) / chunk;
      for (int ph = 0; ph < 4; ++ph) {
        b.off[ph] = bt->ptot[ti][ph];
        bt->ptot[ti][ph] += b.cnt[ph];
        maps[ti][ph].insert(maps[ti][ph].end(), (size_t)b.cnt[ph], i);
      }
    }
  }
  bt->naux = n < nsk_batch::kAux ? n : nsk_batch::kAux;
  if (bt->naux < 2) bt->naux = 0;
  bool aux_ok = bt->naux == 0 || cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int j = 0; j < bt->naux && aux_ok; ++j)
    aux_ok = cudaStreamCreateWithFlags(&bt->aux[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&bt->ev_join[j], cudaEventDisableTiming) == cudaSuccess;
  if (!aux_ok || cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&bt->d_pinst, 2 * sizeof(BatchInst) * n) != cudaSuccess ||
      cudaMalloc(&bt->d_inst, 2 * sizeof(BatchInst) * n) != cudaSuccess ||
      cudaMalloc(&bt->d_bar, 2 * sizeof(unsigned)) != cudaSuccess || cudaMalloc(&bt->d_err, sizeof(int)) != cudaSuccess) {
    nsk_batch_destroy(bt);
    return NSK_ERR_NOMEM;
  }
  for (int ti = 0; ti < 2; ++ti) {
    if (cudaMemcpy(bt->d_inst + (size_t)ti * n, bt->h_inst[ti].data(), sizeof(BatchInst) * n,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(bt->d_pinst + (size_t)ti * n, pinst[ti].data(), sizeof(BatchInst) * n,
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      nsk_batch_destroy(bt);
      return NSK_ERR_CUDA;
    }
    for (int ph = 0; ph < 4; ++ph) {
      const size_t bytes = sizeof(int) * maps[ti][ph].size();
      if (cudaMalloc(&bt->d_blk2inst[ti][ph], bytes) != cudaSuccess ||
          cudaMemcpy(bt->d_blk2inst[ti][ph], maps[ti][ph].data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        nsk_batch_destroy(bt);
        return NSK_ERR_NOMEM;
      }
    }
  }
  if (cudaMemset(bt->d_bar, 0, 2 * sizeof(unsigned)) != cudaSuccess || cudaMemset(bt->d_err, 0, sizeof(int)) != cudaSuccess) {
    nsk_batch_destroy(bt);
    return NSK_ERR_CUDA;
  }
  const int pst = prepare_batch(bt);
  if (pst) {
    nsk_batch_destroy(bt);
    return pst;
  }
  *out = bt;
  return NSK_OK;
}

int nsk_batch_set_schedule(nsk_batch* bt, int tpb, int fused_face, int persistent) {
  if (!bt || (tpb != 128 && tpb != 256) || persistent < 0 || persistent > 2 || fused_face < 0 || fused_face > 5 ||
      fused_face == 3 || (fused_face >= 2 && persistent != 2))
    return NSK_ERR_ARG;
  bt->tpb = tpb;
  bt->fused = fused_face;
  bt->persistent = persistent;
  return NSK_OK;
}

int nsk_batch_get_schedule(nsk_batch* bt, int* tpb, int* fused_face, int* persistent) {
  if (!bt) return NSK_ERR_ARG;
  if (tpb) *tpb = bt->tpb;
  if (fused_face) *fused_face = bt->fused;
  if (persistent) *persistent = bt->persistent;
  return NSK_OK;
}

int nsk_batch_autotune(nsk_batch* bt, int* tpb_out, int* fused_out, int* persistent_out, double* ms_out) {
  const NskRange nvtx_range("nsk_batch_autotune");
  if (!bt) return NSK_ERR_ARG;
  for (nsk_ctx* c : bt->inst)
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  // every instance's own schedule first (the candidate "each instance's own schedule")
  for (nsk_ctx* c : bt->inst) {
    const int r = nsk_autotune(c, nullptr, nullptr, nullptr);
    if (r) return r;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NSK_ERR_CUDA;
  double best = 1e300;
  int bt_tpb = bt->tpb, bt_f = bt->fused, bt_p = bt->persistent, st = NSK_OK;
  const int tpbs[2] = {128, 256};
  for (int per = 0; per < 3 && st == NSK_OK; ++per)
    for (int ti = 0; ti < 2 && st == NSK_OK; ++ti)
      for (int fi = 0; fi < (per == 2 ? 5 : 2) && st == NSK_OK; ++fi) {
        // instance schedule: separate, fused, lean, line, and each instance's own (tuned above)
        const int f = fi == 3 ? 4 : (fi == 4 ? 5 : fi);
        if (f == 5 && ti == 1) continue;  // the instances' own block sizes: one timing
        // warm-up with a prolongation pass (residual: state untouched), then time the stage as a
        // step runs it (rewriting the traces of the unchanged state leaves them as they are; the
        // lean stage as a middle stage of a step: traces read from the trace buffer, the next
        // ones written to the spare buffer)
        st = launch_batch(bt, NSK_MODE_RHS, 0.0, 0.0, tpbs[ti], f, per, 0);
        if (st) break;
        cudaEventRecord(e0, bt->stream);
        for (int r = 0; r < 3 && st == NSK_OK; ++r)
          st = launch_batch(bt, NSK_MODE_RHS, 0.0, 0.0, tpbs[ti], f, per, step_traces(f), false, 2);
        cudaEventRecord(e1, bt->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = NSK_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == NSK_OK && ms / 3.0 < best) {
          best = ms / 3.0;
          bt_tpb = tpbs[ti];
          bt_f = f;
          bt_p = per;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  st = read_error(bt);
  if (st) return st;
  bt->tpb = bt_tpb;
  bt->fused = bt_f;
  bt->persistent = bt_p;
  if (tpb_out) *tpb_out = bt_tpb;
  if (fused_out) *fused_out = bt_f;
  if (persistent_out) *persistent_out = bt_p;
  if (ms_out) *ms_out = best;
  return NSK_OK;
}

int nsk_batch_step(nsk_batch* bt, int nsteps, double cfl, double* step_ms, double* per_instance_latency_ms) {
  const NskRange nvtx_range("nsk_batch_step");
  if (!bt || nsteps < 0) return NSK_ERR_ARG;
  for (nsk_ctx* c : bt->inst)
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return NSK_ERR_CUDA;
  const int dtmode = cfl > 0.0 ? 1 : 0;
  const bool stamps = per_instance_latency_ms != nullptr && nsteps > 0;
  if (stamps) {  // stamp slots and a history of nsteps steps
    if (!bt->d_stamp && cudaMalloc(&bt->d_stamp, sizeof(unsigned long long) * (bt->n + 1)) != cudaSuccess)
      return NSK_ERR_NOMEM;
    if (bt->hist_cap < nsteps) {
      if (bt->d_hist) cudaFree(bt->d_hist);
      bt->d_hist = nullptr;
      bt->hist_cap = 0;
      if (cudaMalloc(&bt->d_hist, sizeof(unsigned long long) * (bt->n + 1) * (size_t)nsteps) != cudaSuccess)
        return NSK_ERR_NOMEM;
      bt->hist_cap = nsteps;
    }
  }
  if (!bt->no_graph &&
      (!bt->graph || bt->graph_tpb != bt->tpb || bt->graph_fused != bt->fused || bt->graph_dtmode != dtmode ||
       bt->graph_persistent != bt->persistent || (dtmode && bt->graph_cfl != cfl) ||
       bt->graph_stamps != (int)stamps || (bt->fused == 5 && bt->graph_inst_sched != inst_schedules(bt)))) {
    destroy_graph(bt);
    cudaGraph_t g;
    if (cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NSK_ERR_CUDA;
    const long long l0 = bt->launches;
    const int st = launch_step(bt, dtmode, cfl, stamps);
    bt->graph_launches = bt->launches - l0;
    bt->launches = l0;  // counted per replay below
    const cudaError_t ce = cudaStreamEndCapture(bt->stream, &g);
    cudaError_t ie = cudaErrorUnknown;
    if (st == NSK_OK && ce == cudaSuccess) {
      ie = cudaGraphInstantiate(&bt->graph, g, 0);
      cudaGraphDestroy(g);
    }
    if (ie != cudaSuccess) {  // capture refused: fall back to direct launches
      cudaGetLastError();
      bt->graph = nullptr;
      bt->no_graph = true;
    }
    bt->graph_tpb = bt->tpb;
    bt->graph_fused = bt->fused;
    bt->graph_dtmode = dtmode;
    bt->graph_persistent = bt->persistent;
    bt->graph_cfl = cfl;
    bt->graph_stamps = (int)stamps;
    bt->graph_inst_sched = inst_schedules(bt);
  }
  if (nsteps > 0 && step_traces(bt->fused)) {  // the traces of the current states, for the first stage
    const int r = launch_prolong(bt, bt->tpb);
    if (r) return r;
  }
  std::vector<cudaEvent_t> ev;
  if (step_ms) {
    ev.resize(nsteps + 1);
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return NSK_ERR_CUDA;
    cudaEventRecord(ev[0], bt->stream);
  }
  const size_t srow = (size_t)(bt->n + 1);
  for (int s = 0; s < nsteps; ++s) {
    if (bt->no_graph) {
      const int r = launch_step(bt, dtmode, cfl, stamps);
      if (r) return r;
    } else {
      if (cudaGraphLaunch(bt->graph, bt->stream) != cudaSuccess) return NSK_ERR_CUDA;
      bt->launches += bt->graph_launches;
    }
    if (step_ms) cudaEventRecord(ev[s + 1], bt->stream);
    if (stamps && cudaMemcpyAsync(bt->d_hist + s * srow, bt->d_stamp, sizeof(unsigned long long) * srow,
                                  cudaMemcpyDeviceToDevice, bt->stream) != cudaSuccess)
      return NSK_ERR_CUDA;
  }
  int st = read_error(bt);
  if (step_ms) {
    for (int s = 0; s < nsteps; ++s) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
      step_ms[s] = ms;
    }
    for (auto& e : ev) cudaEventDestroy(e);
  }
  if (stamps && nsteps > 0) {
    std::vector<unsigned long long> h(srow * (size_t)nsteps);
    if (cudaMemcpy(h.data(), bt->d_hist, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return NSK_ERR_CUDA;
    for (int s = 0; s < nsteps; ++s)
      for (int i = 0; i < bt->n; ++i)
        per_instance_latency_ms[(size_t)s * bt->n + i] = 1e-6 * (double)(h[s * srow + 1 + i] - h[s * srow]);
  }
  return st;
}

long long nsk_batch_launch_count(nsk_batch* bt) { return bt ? bt->launches : -1; }

int nsk_batch_uses_graph(nsk_batch* bt) { return bt ? (bt->graph != nullptr ? 1 : 0) : NSK_ERR_ARG; }

int nsk_batch_set_timeout(nsk_batch* bt, double seconds) {
  if (!bt || !(seconds > 0.0) || seconds > 60.0) return NSK_ERR_ARG;
  bt->timeout_ns = (unsigned long long)(seconds * 1e9);
  destroy_graph(bt);  // the bound is a launch argument baked into the captured graph
  return NSK_OK;
}

int nsk_test_hook_block_batch_barrier(nsk_batch* bt) {
  if (!bt) return NSK_ERR_ARG;
  // arrivals start far above the grid size, so the next barrier can never complete and
  // every block's bounded wait expires
  const unsigned poison[2] = {0x40000000u, 0u};
  if (cudaMemcpyAsync(bt->d_bar, poison, sizeof(poison), cudaMemcpyHostToDevice, bt->stream) != cudaSuccess ||
      cudaStreamSynchronize(bt->stream) != cudaSuccess)
    return NSK_ERR_CUDA;
  return NSK_OK;
}

void nsk_batch_destroy(nsk_batch* bt) {
  if (!bt) return;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  destroy_graph(bt);
  if (bt->d_inst) cudaFree(bt->d_inst);
  if (bt->d_pinst) cudaFree(bt->d_pinst);
  for (int ti = 0; ti < 2; ++ti)
    for (int ph = 0; ph < 4; ++ph)
      if (bt->d_blk2inst[ti][ph]) cudaFree(bt->d_blk2inst[ti][ph]);
  if (bt->d_bar) cudaFree(bt->d_bar);
  if (bt->d_err) cudaFree(bt->d_err);
  if (bt->d_stamp) cudaFree(bt->d_stamp);
  if (bt->d_hist) cudaFree(bt->d_hist);
  for (int j = 0; j < bt->naux; ++j) {
    if (bt->aux[j]) cudaStreamDestroy(bt->aux[j]);
    if (bt->ev_join[j]) cudaEventDestroy(bt->ev_join[j]);
  }
  if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
  if (bt->stream) cudaStreamDestroy(bt->stream);
  delete bt;
}

}  // extern "C"
