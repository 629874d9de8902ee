// Batched persistent stages: many independent 2D scalar DG meshes of uneven size and
// degree advanced together.  One persistent launch per SSP-RK3 stage walks a list of
// 16x8 (or 8x8) cell tiles drawn from every mesh; each tile runs the same fused stage
// (a)-(e) as the single-mesh kernel (scalar_tile), with that mesh's arguments.  The step
// is replayed from a captured CUDA graph, and the launch shape (fused or per-degree
// launches, tile shape, static or counter-driven tile claims, CTAs per SM) is chosen by
// timing every candidate on the batch itself.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dg_scalar_kernel.cuh"

using namespace cvw;

namespace cvw {

struct BatchTile {
  int inst, p, i0, j0;
};

// The reference tabulations of every degree.  With square cells the semi-norm scaling
// (2h/dx)^(2k) and the Gram factors reduce to powers of 2, so one set per degree serves
// all meshes of that degree (only tscale, the vertex-output scaling, depends on h, and
// the RK and residual modes do not read it).
struct AllTables {
  DgTables<2, 1> t1;
  DgTables<2, 2> t2;
  DgTables<2, 3> t3;
  DgTables<2, 4> t4;
};

template <int PSEL>
struct BatchTab {
  using type = DgTables<2, PSEL>;
};
template <>
struct BatchTab<0> {
  using type = AllTables;
};

template <int P>
__device__ __forceinline__ const DgTables<2, P>& pick(const AllTables& T);
template <>
__device__ __forceinline__ const DgTables<2, 1>& pick<1>(const AllTables& T) { return T.t1; }
template <>
__device__ __forceinline__ const DgTables<2, 2>& pick<2>(const AllTables& T) { return T.t2; }
template <>
__device__ __forceinline__ const DgTables<2, 3>& pick<3>(const AllTables& T) { return T.t3; }
template <>
__device__ __forceinline__ const DgTables<2, 4>& pick<4>(const AllTables& T) { return T.t4; }
template <int P>
__device__ __forceinline__ const DgTables<2, P>& pick(const DgTables<2, P>& T) {
  return T;
}

template <int P, int SYS, int TX, int TY, class TT>
__device__ __forceinline__ void batch_tile(const StageArgs& a, const TT& T, const BatchTile& bt, float* smem,
                                           int& cur_p) {
  const DgTables<2, P>& t = pick<P>(T);
  // a new degree needs its tabulations in shared memory; the previous tile's readers
  // have passed the barrier that ends it, and the tile's first barrier publishes them
  if (cur_p != P) {
    stage_tables_to_smem<2, P, TX, TY>(a.tab_img, smem);
    cur_p = P;
  }
  scalar_tile<2, P, SYS, TX, TY>(a, t, bt.i0, bt.j0, smem);
}

template <int TX, int TY>
constexpr size_t batch_smem(int psel) {
  return psel == 1   ? TileLayout<2, 1, TX, TY>::BYTES
         : psel == 2 ? TileLayout<2, 2, TX, TY>::BYTES
         : psel == 3 ? TileLayout<2, 3, TX, TY>::BYTES
         : psel == 4 ? TileLayout<2, 4, TX, TY>::BYTES
                     : std::max(std::max(TileLayout<2, 1, TX, TY>::BYTES, TileLayout<2, 2, TX, TY>::BYTES),
                                std::max(TileLayout<2, 3, TX, TY>::BYTES, TileLayout<2, 4, TX, TY>::BYTES));
}

// Persistent stage over tiles[0..ntiles).  PSEL = 0: tiles of any degree (switch per
// tile); PSEL = p: every tile has degree p.  sched == nullptr: CTA b takes tiles
// b, b + G, b + 2G, ...; otherwise sched[0] is the next unclaimed tile and sched[1]
// counts CTAs that have left -- the last one resets both for the next launch in stream
// order.  No CTA ever waits on another.
// Register caps (CTAs per SM at 128 threads) at the single-mesh kernels' allocation:
// without them the per-tile argument loads and the degree switch inflate the fused
// kernel to the 255-register ceiling.
template <int PSEL, int TX, int TY>
constexpr int batch_min_ctas() {
  return (PSEL == 0 || PSEL == 4 ? 3 : PSEL == 3 ? 4 : PSEL == 2 ? 6 : 8) * (128 / (TX * TY));
}

template <int PSEL, int SYS, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (batch_min_ctas<PSEL, TX, TY>()))
    dg_scalar_batch(const BatchTile* __restrict__ tiles, int ntiles, const StageArgs* __restrict__ args,
                    int* __restrict__ sched, const __grid_constant__ typename BatchTab<PSEL>::type T) {
  extern __shared__ __align__(16) float smem[];
  __shared__ StageArgs sa;
  __shared__ BatchTile s_bt;
  constexpr int NW = (int)(sizeof(StageArgs) / sizeof(int));
  static_assert(sizeof(StageArgs) % sizeof(int) == 0, "StageArgs copied as words");
  int cur_p = 0;
  int t = blockIdx.x;
  for (;;) {
    // warp 0 claims the tile and copies its mesh's arguments; one barrier publishes both
    if (threadIdx.x < 32) {
      int tt = t;
      if (sched) {
        if (threadIdx.x == 0) tt = atomicAdd(sched, 1);
        tt = __shfl_sync(0xffffffffu, tt, 0);
      }
      if (tt < ntiles) {
        const BatchTile bt = tiles[tt];
        const int* src = reinterpret_cast<const int*>(args + bt.inst);
        int* dst = reinterpret_cast<int*>(&sa);
        for (int k = threadIdx.x; k < NW; k += 32) dst[k] = src[k];
        if (threadIdx.x == 0) s_bt = bt;
      } else if (threadIdx.x == 0) {
        s_bt.inst = -1;
      }
    }
    __syncthreads();
    const BatchTile bt = s_bt;
    if (bt.inst < 0) break;
    if constexpr (PSEL != 0) {
      batch_tile<PSEL, SYS, TX, TY>(sa, T, bt, smem, cur_p);
    } else {
      switch (bt.p) {
        case 1: batch_tile<1, SYS, TX, TY>(sa, T, bt, smem, cur_p); break;
        case 2: batch_tile<2, SYS, TX, TY>(sa, T, bt, smem, cur_p); break;
        case 3: batch_tile<3, SYS, TX, TY>(sa, T, bt, smem, cur_p); break;
        default: batch_tile<4, SYS, TX, TY>(sa, T, bt, smem, cur_p); break;
      }
    }
    __syncthreads();  // the next tile overwrites sa, s_bt and the shared tile
    t += gridDim.x;
  }
  if (sched && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
      sched[0] = 0;
      sched[1] = 0;
    }
  }
}

}  // namespace cvw

namespace {

constexpr int kBatchSlots = 4;      // argument sets: RK stages 0..2, residual
constexpr int kSlotResidual = 3;
constexpr int kNumTiles = 2;        // 16x8, 8x8
constexpr int kSchedCounters = 5;   // fused launch + one per degree

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

struct TileShape {
  int tx, ty;
};
constexpr TileShape kTiles[kNumTiles] = {{16, 8}, {8, 8}};

// Type-erased launcher of one kernel instantiation.
struct KernelRef {
  const void* fn;
  size_t smem;
};

template <int PSEL, int TX, int TY>
KernelRef kref() {
  return KernelRef{(const void*)dg_scalar_batch<PSEL, CVWENO_BURGERS, TX, TY>, batch_smem<TX, TY>(PSEL)};
}

KernelRef kernel_for(int tile, int psel) {
  if (tile == 0) {
    switch (psel) {
      case 0: return kref<0, 16, 8>();
      case 1: return kref<1, 16, 8>();
      case 2: return kref<2, 16, 8>();
      case 3: return kref<3, 16, 8>();
      default: return kref<4, 16, 8>();
    }
  }
  switch (psel) {
    case 0: return kref<0, 8, 8>();
    case 1: return kref<1, 8, 8>();
    case 2: return kref<2, 8, 8>();
    case 3: return kref<3, 8, 8>();
    default: return kref<4, 8, 8>();
  }
}

}  // namespace

struct cvweno_batch_s {
  int device = 0;
  int count = 0;
  int sm_count = 0;
  std::vector<cvweno_mesh> meshes;
  std::vector<int64_t> offsets;
  AllTables* tables = nullptr;  // host
  int have_p[cvw::kMaxP + 1] = {0};
  cvweno_batch_plan plan;
  // tile list of the current tile shape, sorted by degree (4 first)
  BatchTile* d_tiles = nullptr;
  int ntiles = 0;
  int seg_off[cvw::kMaxP + 1] = {0}, seg_cnt[cvw::kMaxP + 1] = {0};
  int tiles_shape = -1;
  // per-instance stage arguments [slot][count] (device) and their host image
  StageArgs* d_args = nullptr;
  std::vector<StageArgs> h_args;
  std::vector<bool> slot_valid;
  const float* slot_u[kBatchSlots] = {nullptr};
  const float* slot_out[kBatchSlots] = {nullptr};
  std::vector<double> slot_dt;
  int occ[kNumTiles][cvw::kMaxP + 1] = {{0}};  // resident CTAs per SM of each kernel
  int* d_sched = nullptr;   // [kSchedCounters][2]
  int* d_status = nullptr;  // [count]
  int* h_status = nullptr;  // pinned [count]
  cudaStream_t side[cvw::kMaxP + 1] = {nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[cvw::kMaxP + 1] = {nullptr};
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  float* graph_u = nullptr;
  cvweno_batch_plan graph_plan;
};

namespace {

cvweno_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CVWENO_OK : CVWENO_ERR_CUDA; }

bool plan_valid(const cvweno_batch_plan& p) {
  return (p.schedule == CVWENO_BATCH_FUSED || p.schedule == CVWENO_BATCH_GROUPED) && p.tile >= 0 &&
         p.tile < kNumTiles && (p.dynamic == 0 || p.dynamic == 1) && p.ctas_per_sm >= 0 && p.ctas_per_sm <= 32 &&
         (p.use_graph == 0 || p.use_graph == 1);
}

bool same_shape(const cvweno_batch_plan& a, const cvweno_batch_plan& b) {
  return a.schedule == b.schedule && a.tile == b.tile && a.dynamic == b.dynamic && a.ctas_per_sm == b.ctas_per_sm;
}

void drop_graph(cvweno_batch b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_u = nullptr;
}

// Tile list of shape `tile`: every instance's tiles, degree 4 first (heaviest work
// first keeps the counter-driven claims balanced), instances in order, tiles row-major.
cvweno_status build_tiles(cvweno_batch b, int tile) {
  if (b->tiles_shape == tile) return CVWENO_OK;
  const int tx = kTiles[tile].tx, ty = kTiles[tile].ty;
  std::vector<BatchTile> list;
  for (int p = cvw::kMaxP; p >= 1; --p) {
    b->seg_off[p] = (int)list.size();
    for (int k = 0; k < b->count; ++k) {
      const cvweno_mesh m = b->meshes[k];
      if (m->p != p) continue;
      for (int j0 = 0; j0 < m->ny; j0 += ty)
        for (int i0 = 0; i0 < m->nx; i0 += tx) list.push_back(BatchTile{k, p, i0, j0});
    }
    b->seg_cnt[p] = (int)list.size() - b->seg_off[p];
  }
  if (list.size() > (size_t)INT32_MAX / 2) return CVWENO_ERR_ARG;
  if (b->d_tiles) cudaFree(b->d_tiles);
  b->d_tiles = nullptr;
  b->tiles_shape = -1;
  if (cudaMalloc(&b->d_tiles, sizeof(BatchTile) * list.size()) != cudaSuccess) return CVWENO_ERR_NOMEM;
  if (cudaMemcpy(b->d_tiles, list.data(), sizeof(BatchTile) * list.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return CVWENO_ERR_CUDA;
  b->ntiles = (int)list.size();
  b->tiles_shape = tile;
  return CVWENO_OK;
}

// Argument set `slot` for state u (RK stages 0..2 read u_n = u; the residual slot
// writes out).  Uploaded only when the pointers or the step sizes change.
cvweno_status set_slot_args(cvweno_batch b, int slot, const float* in_u, float* out, const double* dt,
                            cudaStream_t s) {
  bool same = b->slot_valid[slot] && b->slot_u[slot] == in_u && b->slot_out[slot] == out;
  if (same && dt)
    for (int k = 0; k < b->count && same; ++k) same = b->slot_dt[(size_t)slot * b->count + k] == dt[k];
  if (same) return CVWENO_OK;
  static const float ra[3] = {0.0f, 0.75f, 1.0f / 3.0f}, rb[3] = {1.0f, 0.25f, 2.0f / 3.0f};
  for (int k = 0; k < b->count; ++k) {
    const cvweno_mesh m = b->meshes[k];
    StageArgs a = stage_base_args(m);
    a.status = b->d_status + k;
    float* uk = const_cast<float*>(in_u) + b->offsets[k];
    if (slot == kSlotResidual) {
      a.u_in = uk;
      a.u_n = uk;
      a.u_out = out + b->offsets[k];
      a.mode = kModeResidual;
    } else {
      a.u_in = slot == 0 ? uk : slot == 1 ? m->d_u1 : m->d_u2;
      a.u_n = uk;
      a.u_out = slot == 0 ? m->d_u1 : slot == 1 ? m->d_u2 : uk;
      a.rk_a = ra[slot];
      a.rk_b = rb[slot];
      a.dt = (float)dt[k];
      a.mode = kModeRK;
      b->slot_dt[(size_t)slot * b->count + k] = dt[k];
    }
    b->h_args[(size_t)slot * b->count + k] = a;
  }
  // pageable source: the copy has read it when the call returns
  cudaError_t e = cudaMemcpyAsync(b->d_args + (size_t)slot * b->count, b->h_args.data() + (size_t)slot * b->count,
                                  sizeof(StageArgs) * b->count, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  b->slot_valid[slot] = true;
  b->slot_u[slot] = in_u;
  b->slot_out[slot] = out;
  return CVWENO_OK;
}

cudaError_t launch_one(cvweno_batch b, int psel, int slot, cudaStream_t s) {
  const cvweno_batch_plan& pl = b->plan;
  const KernelRef k = kernel_for(pl.tile, psel);
  const int off = psel ? b->seg_off[psel] : 0, cnt = psel ? b->seg_cnt[psel] : b->ntiles;
  if (cnt == 0) return cudaSuccess;
  const int nthr = kTiles[pl.tile].tx * kTiles[pl.tile].ty;
  const int occ = b->occ[pl.tile][psel];
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int per_sm = pl.ctas_per_sm > 0 ? std::min(pl.ctas_per_sm, occ) : occ;
  const int grid = std::min(cnt, per_sm * b->sm_count);
  const BatchTile* tiles = b->d_tiles + off;
  const StageArgs* args = b->d_args + (size_t)slot * b->count;
  int* sched = pl.dynamic ? b->d_sched + 2 * psel : nullptr;
  void* params[5] = {(void*)&tiles, (void*)&cnt, (void*)&args, (void*)&sched, nullptr};
  switch (psel) {
    case 0: params[4] = (void*)b->tables; break;
    case 1: params[4] = (void*)&b->tables->t1; break;
    case 2: params[4] = (void*)&b->tables->t2; break;
    case 3: params[4] = (void*)&b->tables->t3; break;
    default: params[4] = (void*)&b->tables->t4; break;
  }
  return cudaLaunchKernel(k.fn, dim3(grid), dim3(nthr), params, k.smem, s);
}

// One stage of every instance with argument set `slot`.
cudaError_t enqueue_stage(cvweno_batch b, int slot, cudaStream_t s) {
  if (b->plan.schedule == CVWENO_BATCH_FUSED) return launch_one(b, 0, slot, s);
  cudaError_t e = cudaEventRecord(b->ev_fork, s);
  for (int p = cvw::kMaxP; p >= 1 && e == cudaSuccess; --p) {
    if (!b->seg_cnt[p]) continue;
    e = cudaStreamWaitEvent(b->side[p], b->ev_fork, 0);
    if (e == cudaSuccess) e = launch_one(b, p, slot, b->side[p]);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[p], b->side[p]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[p], 0);
  }
  return e;
}

cudaError_t enqueue_step(cvweno_batch b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int st = 0; st < 3 && e == cudaSuccess; ++st) e = enqueue_stage(b, st, s);
  return e;
}

void free_batch(cvweno_batch b) {
  drop_graph(b);
  for (cvweno_mesh m : b->meshes)
    if (m) cvweno_mesh_destroy(m);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_args) cudaFree(b->d_args);
  if (b->d_sched) cudaFree(b->d_sched);
  if (b->d_status) cudaFree(b->d_status);
  if (b->h_status) cudaFreeHost(b->h_status);
  for (int p = 0; p <= cvw::kMaxP; ++p) {
    if (b->side[p]) cudaStreamDestroy(b->side[p]);
    if (b->ev_join[p]) cudaEventDestroy(b->ev_join[p]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  free(b->tables);
  delete b;
}

template <int P>
bool same_tables(const DgTables<2, P>& x, const DgTables<2, P>& y) {
  // everything but tscale (vertex-output scaling, not read by the batch)
  DgTables<2, P> a = x, c = y;
  memset(a.tscale, 0, sizeof(a.tscale));
  memset(c.tscale, 0, sizeof(c.tscale));
  return memcmp(&a, &c, sizeof(a)) == 0;
}

template <int P>
bool take_tables(DgTables<2, P>& dst, bool have, const cvweno_mesh m) {
  const DgTables<2, P>& src = *static_cast<const DgTables<2, P>*>(m->tables);
  if (!have) {
    dst = src;
    return true;
  }
  return same_tables<P>(dst, src);
}

}  // namespace

extern "C" {

cvweno_status cvweno_batch_create(const cvweno_mesh_desc* descs, int count, cvweno_batch* out) {
  if (!descs || !out || count < 1 || count > (1 << 20)) return CVWENO_ERR_ARG;
  *out = nullptr;
  for (int k = 0; k < count; ++k) {
    const cvweno_mesh_desc& d = descs[k];
    if (d.dim != 2 || d.kind != CVWENO_DG) return CVWENO_ERR_UNSUPPORTED;
    if (d.system != CVWENO_BURGERS || d.params.hweno_limiter) return CVWENO_ERR_UNSUPPORTED;
    if (d.nx < 1 || d.ny < 1) return CVWENO_ERR_ARG;
    const double dx = (d.x1 - d.x0) / d.nx, dy = (d.y1 - d.y0) / d.ny;
    if (!(fabs(dx - dy) <= 1e-12 * fabs(dx))) return CVWENO_ERR_ARG;
  }
  cvweno_batch b = new (std::nothrow) cvweno_batch_s;
  if (!b) return CVWENO_ERR_NOMEM;
  b->count = count;
  cvweno_status st = CVWENO_OK;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return CVWENO_ERR_CUDA;
  }
  b->tables = (AllTables*)calloc(1, sizeof(AllTables));
  if (!b->tables) {
    delete b;
    return CVWENO_ERR_NOMEM;
  }
  b->offsets.assign(count + 1, 0);
  b->meshes.assign(count, nullptr);
  for (int k = 0; k < count && st == CVWENO_OK; ++k) {
    st = cvweno_mesh_create(&descs[k], &b->meshes[k]);
    if (st != CVWENO_OK) break;
    const cvweno_mesh m = b->meshes[k];
    b->offsets[k + 1] = b->offsets[k] + m->nstate;
    bool ok = true;
    switch (m->p) {
      case 1: ok = take_tables<1>(b->tables->t1, b->have_p[1], m); break;
      case 2: ok = take_tables<2>(b->tables->t2, b->have_p[2], m); break;
      case 3: ok = take_tables<3>(b->tables->t3, b->have_p[3], m); break;
      case 4: ok = take_tables<4>(b->tables->t4, b->have_p[4], m); break;
      default: ok = false;
    }
    if (!ok) st = CVWENO_ERR_ARG;  // parameters that change the tabulations
    b->have_p[m->p] = 1;
  }
  if (st == CVWENO_OK) {
    b->h_args.assign((size_t)kBatchSlots * count, StageArgs{});
    b->slot_valid.assign(kBatchSlots, false);
    b->slot_dt.assign((size_t)kBatchSlots * count, 0.0);
    e = cudaMalloc(&b->d_args, sizeof(StageArgs) * kBatchSlots * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sched, sizeof(int) * 2 * kSchedCounters);
    if (e == cudaSuccess) e = cudaMemset(b->d_sched, 0, sizeof(int) * 2 * kSchedCounters);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int) * count);
    for (int p = 0; p <= cvw::kMaxP && e == cudaSuccess; ++p) {
      e = cudaStreamCreateWithFlags(&b->side[p], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[p], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    // shared-memory opt-in and occupancy of every kernel, once (not capturable calls)
    for (int t = 0; t < kNumTiles && e == cudaSuccess; ++t)
      for (int ps = 0; ps <= cvw::kMaxP && e == cudaSuccess; ++ps) {
        const KernelRef k = kernel_for(t, ps);
        if (k.smem > 48 * 1024)
          e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ[t][ps], k.fn, kTiles[t].tx * kTiles[t].ty,
                                                            k.smem);
      }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = CVWENO_ERR_CUDA;
  }
  if (st == CVWENO_OK) {
    b->plan = cvweno_batch_plan{CVWENO_BATCH_FUSED, 0, 1, 0, 1, 0.0f};
    st = build_tiles(b, b->plan.tile);
  }
  if (st != CVWENO_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return CVWENO_OK;
}

cvweno_status cvweno_batch_destroy(cvweno_batch b) {
  if (!b) return CVWENO_ERR_ARG;
  cudaDeviceSynchronize();
  free_batch(b);
  return CVWENO_OK;
}

cvweno_status cvweno_batch_offsets(cvweno_batch b, int64_t* offsets) {
  if (!b || !offsets) return CVWENO_ERR_ARG;
  for (int k = 0; k <= b->count; ++k) offsets[k] = b->offsets[k];
  return CVWENO_OK;
}

cvweno_status cvweno_batch_set_plan(cvweno_batch b, const cvweno_batch_plan* plan) {
  if (!b || !plan || !plan_valid(*plan)) return CVWENO_ERR_ARG;
  cvweno_status st = build_tiles(b, plan->tile);
  if (st != CVWENO_OK) return st;
  b->plan = *plan;
  return CVWENO_OK;
}

cvweno_status cvweno_batch_get_plan(cvweno_batch b, cvweno_batch_plan* plan) {
  if (!b || !plan) return CVWENO_ERR_ARG;
  *plan = b->plan;
  return CVWENO_OK;
}

cvweno_status cvweno_batch_residual(cvweno_batch b, const float* u, float* dudt, void* stream) {
  cvw::NvtxRange range("cvweno_batch_residual");
  if (!b || !u || !dudt || u == dudt) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  cvweno_status st = set_slot_args(b, kSlotResidual, u, dudt, nullptr, s);
  if (st != CVWENO_OK) return st;
  return cuda_status(enqueue_stage(b, kSlotResidual, s));
}

cvweno_status cvweno_batch_advance(cvweno_batch b, float* u, const double* dt, int nsteps, void* stream) {
  cvw::NvtxRange range("cvweno_batch_advance");
  if (!b || !u || !dt || nsteps < 0) return CVWENO_ERR_ARG;
  for (int k = 0; k < b->count; ++k)
    if (!(dt[k] > 0.0)) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  for (int st = 0; st < 3; ++st) {
    cvweno_status r = set_slot_args(b, st, u, u, dt, s);
    if (r != CVWENO_OK) return r;
  }
  if (!b->plan.use_graph) {
    for (int i = 0; i < nsteps; ++i) {
      cudaError_t e = enqueue_step(b, s);
      if (e != cudaSuccess) return CVWENO_ERR_CUDA;
    }
    return CVWENO_OK;
  }
  if (b->graph && (b->graph_u != u || !same_shape(b->graph_plan, b->plan))) drop_graph(b);
  if (!b->graph && nsteps > 0) {
    // the step reads its arguments from device memory, so only the state pointer and
    // the launch shape are baked into the graph
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return CVWENO_ERR_CUDA;
    cudaError_t el = enqueue_step(b, b->cap);
    e = cudaStreamEndCapture(b->cap, &g);
    if (el != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return CVWENO_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return CVWENO_ERR_CUDA;
    }
    b->graph_u = u;
    b->graph_plan = b->plan;
  }
  for (int i = 0; i < nsteps; ++i)
    if (cudaGraphLaunch(b->graph, s) != cudaSuccess) return CVWENO_ERR_CUDA;
  return CVWENO_OK;
}

cvweno_status cvweno_batch_autotune(cvweno_batch b, const float* u, cvweno_batch_plan* best, void* stream) {
  if (!b || !u) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  const cvweno_batch_plan keep = b->plan;
  // the residual pass writes to the first instance-sized stage buffers of the meshes:
  // build a scratch output pointer per instance through the residual slot's arguments
  cvweno_status st = CVWENO_OK;
  std::vector<StageArgs> tmp(b->count);
  for (int k = 0; k < b->count; ++k) {
    const cvweno_mesh m = b->meshes[k];
    StageArgs a = stage_base_args(m);
    a.status = b->d_status + k;
    a.u_in = const_cast<float*>(u) + b->offsets[k];
    a.u_n = a.u_in;
    a.u_out = m->d_u1;
    a.mode = kModeResidual;
    tmp[k] = a;
  }
  if (cudaMemcpy(b->d_args + (size_t)kSlotResidual * b->count, tmp.data(), sizeof(StageArgs) * b->count,
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return CVWENO_ERR_CUDA;
  b->slot_valid[kSlotResidual] = false;  // the residual slot now holds the scratch set
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return CVWENO_ERR_CUDA;
  }
  cvweno_batch_plan win = keep;
  float win_ms = 1e30f;
  const int cps_options[3] = {0, 2, 1};
  for (int sch = 0; sch < 2 && st == CVWENO_OK; ++sch)
    for (int tile = 0; tile < kNumTiles && st == CVWENO_OK; ++tile)
      for (int dyn = 0; dyn < 2 && st == CVWENO_OK; ++dyn)
        for (int c = 0; c < 3 && st == CVWENO_OK; ++c) {
          cvweno_batch_plan cand{sch, tile, dyn, cps_options[c], keep.use_graph, 0.0f};
          st = build_tiles(b, tile);
          if (st != CVWENO_OK) break;
          b->plan = cand;
          cudaError_t e = enqueue_stage(b, kSlotResidual, s);  // warm-up
          const int reps = 3;
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          for (int r = 0; r < reps && e == cudaSuccess; ++r) e = enqueue_stage(b, kSlotResidual, s);
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            st = CVWENO_ERR_CUDA;
            break;
          }
          ms /= reps;
          if (ms < win_ms) {
            win_ms = ms;
            win = cand;
            win.ms = ms;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CVWENO_OK) {
    b->plan = keep;
    build_tiles(b, keep.tile);
    return st;
  }
  st = build_tiles(b, win.tile);
  if (st != CVWENO_OK) return st;
  b->plan = win;
  if (best) *best = win;
  return CVWENO_OK;
}

cvweno_status cvweno_batch_status_check(cvweno_batch b, int* first_bad, void* stream) {
  if (!b) return CVWENO_ERR_ARG;
  cudaStream_t s = S(stream);
  if (first_bad) *first_bad = -1;
  cudaError_t e = cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  int all = 0, bad = -1;
  for (int k = 0; k < b->count; ++k) {
    all |= b->h_status[k];
    if (b->h_status[k] && bad < 0) bad = k;
  }
  if (first_bad) *first_bad = bad;
  if (all) {
    e = cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->count, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CVWENO_ERR_CUDA;
  }
  if (all & kStatCheck) return CVWENO_ERR_CHECK;
  if (all & kStatPositivity) return CVWENO_ERR_POSITIVITY;
  if (all & kStatNonfinite) return CVWENO_ERR_NONFINITE;
  if (all & kStatTimeout) return CVWENO_ERR_TIMEOUT;
  return CVWENO_OK;
}

}  // extern "C"
