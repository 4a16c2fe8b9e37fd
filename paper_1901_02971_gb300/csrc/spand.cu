// C-ABI entry points, device memory management, the level scheduler of the
// numeric factorization (Algorithm 2) and the PCG driver (Sec. 4).
#include "spand.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <numeric>
#include <stdexcept>
#include <string>
#include <climits>
#include <functional>
#include <map>
#include <tuple>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cpqr_cluster.cuh"
#include "cpqr_reg.cuh"
#include "factor_kernels.cuh"
#include "schur_tc.cuh"
#include "schur_tma.cuh"
#include "sparsify_interp.cuh"
#include "sparsify_rand.cuh"
#include "sparsify_sim.cuh"
#include "sketch.cuh"
#include "solve_kernels.cuh"
#include "spand_internal.h"

namespace spand {

thread_local std::string g_err;

struct Fail {
  int code;
  std::string msg;
};

#define CK(expr)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      throw Fail{e_ == cudaErrorMemoryAllocation ? SPAND_ERR_OOM : SPAND_ERR_CUDA,            \
                 std::string(#expr) + ": " + cudaGetErrorString(e_)};                         \
  } while (0)

#define CKLAUNCH() CK(cudaGetLastError())

static inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// Leading dimension of a cluster's block row: its size rounded up to 4
// elements, so that every block's columns start on a 16-byte boundary (vector
// loads in the tensor-core Schur update); the padding rows stay zero.  Used by
// the analysis (assembly offsets) and every layout.
static inline int32_t row_ld(int32_t size) { return (std::max<int32_t>(size, 1) + 3) / 4 * 4; }

constexpr size_t kCpqrChunkBudget = 224 * 1024;  // shared memory per sparsification CTA (chunk included)
constexpr size_t kSmemPerSM = 228 * 1024;        // shared memory of one SM (each resident CTA also reserves 1 KB)
constexpr int kCpqrMaxCluster = 8;              // thread-block cluster size (broadcasts to 16 CTAs cost 3.5x more)
constexpr int kAuxStreams = 8;
constexpr int kApplyCtasPerSm = 4;  // the most CTAs per SM the apply autotuner tries

// Chunked bump allocator over cudaMalloc; reset() keeps the chunks for reuse.
class DevArena {
  struct Chunk {
    char* p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks_;
  size_t cur_ = 0;

 public:
  size_t bytes_held = 0;
  void* alloc(size_t bytes) {
    bytes = align256(std::max<size_t>(bytes, 1));
    while (cur_ < chunks_.size()) {
      Chunk& c = chunks_[cur_];
      if (c.used + bytes <= c.cap) {
        void* p = c.p + c.used;
        c.used += bytes;
        return p;
      }
      ++cur_;
    }
    size_t cap = std::max<size_t>(bytes, size_t(64) << 20);
    char* p = nullptr;
    CK(cudaMalloc(&p, cap));
    chunks_.push_back({p, cap, bytes});
    bytes_held += cap;
    cur_ = chunks_.size() - 1;
    return p;
  }
  void reset() {
    for (auto& c : chunks_) c.used = 0;
    cur_ = 0;
  }
  void release() {
    for (auto& c : chunks_) cudaFree(c.p);
    chunks_.clear();
    cur_ = 0;
    bytes_held = 0;
  }
  ~DevArena() { release(); }
};

// Pinned host staging for descriptor uploads: cudaMemcpyAsync from pinned
// memory returns at once, so the host keeps building the next launches while
// the copies wait for their turn in the stream.  reset() may only be called
// once the stream has executed every copy taken from the arena.
class PinnedStage {
  struct Chunk {
    char* p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks_;
  size_t cur_ = 0;

 public:
  void* take(size_t bytes) {
    bytes = align256(std::max<size_t>(bytes, 1));
    while (cur_ < chunks_.size()) {
      Chunk& c = chunks_[cur_];
      if (c.used + bytes <= c.cap) {
        void* p = c.p + c.used;
        c.used += bytes;
        return p;
      }
      ++cur_;
    }
    size_t cap = std::max<size_t>(bytes, size_t(16) << 20);
    char* p = nullptr;
    CK(cudaMallocHost(&p, cap));
    chunks_.push_back({p, cap, bytes});
    cur_ = chunks_.size() - 1;
    return p;
  }
  void reset() {
    for (auto& c : chunks_) c.used = 0;
    cur_ = 0;
  }
  ~PinnedStage() {
    for (auto& c : chunks_) cudaFreeHost(c.p);
  }
};

// Grow-only contiguous device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  void* ensure(size_t bytes) {
    if (bytes <= cap && p) return p;
    if (p) {
      CK(cudaDeviceSynchronize());
      cudaFree(p);
      p = nullptr;
      cap = 0;
    }
    size_t c = align256(std::max<size_t>(bytes + bytes / 4, 256));
    CK(cudaMalloc(&p, c));
    cap = c;
    return p;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  ~DevBuf() { release(); }
};

// Host-side packer for one upload of descriptor arrays.
// It records each array's place (256-byte aligned) without copying, and
// write() copies them straight into the destination (the pinned staging
// buffer): no intermediate host buffer is allocated, zero-filled and copied
// again (at the leaf level the apply program alone is several MB per step).
// The arrays must stay alive and unchanged until write().
struct Packer {
  struct Part {
    const void* p;
    size_t off, bytes;
  };
  std::vector<Part> parts;
  size_t size = 0;
  template <typename X>
  size_t add(const std::vector<X>& v) {
    const size_t off = align256(size), bytes = v.size() * sizeof(X);
    if (bytes) parts.push_back({v.data(), off, bytes});
    size = off + bytes;
    return off;
  }
  bool empty() const { return size == 0; }
  void write(void* dst) const {
    for (const Part& q : parts) std::memcpy((char*)dst + q.off, q.p, q.bytes);
  }
};

template <typename TF>
struct ApplyStep {
  int n_elim = 0, n_sq = 0;
  const ElimOp<TF>* elim = nullptr;
  const SqOp<TF>* sq = nullptr;
  const int32_t* slots = nullptr;
  // per-CTA work items of the split elimination GEMVs
  int n_fy = 0, n_fu = 0, n_ba = 0, n_bx = 0;
  const ApplyItem *fy = nullptr, *fu = nullptr, *ba = nullptr, *bx = nullptr;
  // forward scatter: [0, nassign) assignments x_s = y_s, then subtractions
  int64_t ntgt = 0, nassign = 0;
  const int32_t* tslot = nullptr;
  const int64_t* tptr = nullptr;
  const int64_t* tidx = nullptr;
  size_t sm_ns = 0, sm_m = 0, sm_np = 0, sm_r = 0;
  // per-CTA work items of the scaling + coarse-basis GEMVs
  int n_sy = 0, n_sc = 0, n_sz = 0, n_sx = 0;
  const ApplyItem *sy = nullptr, *sc = nullptr, *sz = nullptr, *sx = nullptr;
};

// Process-wide caches of device attributes and of the kernel attributes set so
// far, keyed by device: handles on different host threads (or devices) share
// them, so every access holds g_attr_mutex.
static std::mutex g_attr_mutex;

static int current_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  return dev;
}

// Streaming multiprocessors of the current device.
static int num_sms() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  static std::unordered_map<int, int> cached;
  auto it = cached.find(dev);
  if (it != cached.end()) return it->second;
  int n = 0;
  CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  cached[dev] = n;
  return n;
}

// Clusters of more than 8 CTAs need an explicit opt-in per kernel.
static void ensure_nonportable_cluster(const void* fn) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  static std::unordered_map<const void*, std::vector<int>> done;
  auto& devs = done[fn];
  if (std::find(devs.begin(), devs.end(), dev) != devs.end()) return;
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  devs.push_back(dev);
}

// Highest dynamic shared memory requested so far, per kernel and device.
static void ensure_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  static std::unordered_map<const void*, std::unordered_map<int, size_t>> done;
  size_t& have = done[fn][dev];
  if (have >= bytes) return;
  CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
}

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime
// (no link against the driver library); nullptr if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn tmap_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

// Tensor map over a column-major FP32 block row (ld floats between columns,
// rows x cols), boxes of 32 rows x box_cols columns, 128-byte swizzle,
// zeros outside.  False if the driver refuses it.
static bool encode_row_map(CUtensorMap* m, const float* base, int rows, int cols, int ld, int box_cols) {
  EncodeTiledFn enc = tmap_encoder();
  if (!enc || rows <= 0 || cols <= 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {32u, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static std::mutex g_cluster_mutex;  // guards the cached cluster-size probe

// Largest cluster size (16 or 8) at which the sparsification kernel can be
// resident with a full shared-memory chunk on this device.
template <typename T>
static int cpqr_max_cluster() {
  if constexpr (kCpqrMaxCluster <= 8) return kCpqrMaxCluster;
  std::lock_guard<std::mutex> lk(g_cluster_mutex);
  static int cached[2] = {0, 0};
  int& c = cached[sizeof(T) == 8 ? 1 : 0];
  if (c) return c;
  const void* fn = (const void*)k_cpqr_cluster<T, true, 256>;
  const size_t smem = kCpqrChunkBudget;
  ensure_smem(fn, smem);
  c = 8;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0) c = 16;
  }
  cudaGetLastError();  // a refused query only means 8
  return c;
}


// Kernel-family profiler: launch counts always; with profiling on, a CUDA
// event pair on the launching stream around each batch of launches of one
// family, plus its algorithmic flops and bytes.
enum Family { F_POTRF = 0, F_TRSM, F_SCHUR, F_CPQR, F_COPY, F_APPLY, F_PCG, F_NFAM };

struct KProf {
  bool on = false;
  int64_t launches = 0;
  double ms[F_NFAM] = {}, flops[F_NFAM] = {}, bytes[F_NFAM] = {};
  int64_t count[F_NFAM] = {};
  struct Pend {
    int fam;
    cudaEvent_t a, b;
    double flops, bytes;
    int64_t nl;
  };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  int begin(int fam, cudaStream_t s) {
    if (!on) return -1;
    Pend p{fam, get(), get(), 0.0, 0.0, 0};
    CK(cudaEventRecord(p.a, s));
    pend.push_back(p);
    return (int)pend.size() - 1;
  }
  void end(int id, cudaStream_t s, double flops, double bytes, int64_t nl) {
    if (id < 0) return;
    Pend& p = pend[id];
    p.flops += flops;
    p.bytes += bytes;
    p.nl += nl;
    CK(cudaEventRecord(p.b, s));
  }
  void add(int id, double flops, double bytes) {
    if (id < 0) return;
    pend[id].flops += flops;
    pend[id].bytes += bytes;
  }
  void flush() {  // call after a synchronisation point
    for (auto& p : pend) {
      float t = 0;
      CK(cudaEventSynchronize(p.b));
      CK(cudaEventElapsedTime(&t, p.a, p.b));
      ms[p.fam] += t;
      flops[p.fam] += p.flops;
      bytes[p.fam] += p.bytes;
      count[p.fam] += p.nl;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pend.clear();
  }
  void reset() {
    for (int f = 0; f < F_NFAM; ++f) ms[f] = flops[f] = bytes[f] = 0, count[f] = 0;
  }
  ~KProf() {
    for (auto& p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace spand

using namespace spand;

// Host arrays handed back after use and reused by later steps and
// factorizations: the apply program's per-step arrays run to megabytes at
// the leaf level, and fresh allocations of that size pay first-touch page
// faults on every factorization.
template <typename X>
struct VecPool {
  std::vector<std::vector<X>> free;
  std::vector<X> take() {
    if (free.empty()) return {};
    std::vector<X> v = std::move(free.back());
    free.pop_back();
    v.clear();
    return v;
  }
  void give(std::vector<X>&& v) {
    if (v.capacity() && free.size() < 64) free.push_back(std::move(v));
  }
};

struct spand_handle_s {
  spand_opts opts{};
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<double> vals;
  Tree tree;
  // step-1 assembly: original nnz e -> (cluster row, offset in that row)
  std::vector<int32_t> asm_row;
  std::vector<int64_t> asm_off;
  // envelope of the step-1 pivot blocks (pieces of A itself; other pivots
  // are dense): per initial cluster, U's tile bandwidth (0 = dense), the
  // Cholesky flops sum_j r_j^2 over U's row lengths r_j, and nnz(U)
  std::vector<int32_t> env_bw, env_bw32;  // in 64-tiles and in 32-tiles
  std::vector<int32_t> env_band;          // element half-bandwidth max_i (i - f(i)) (0 = dense)
  std::vector<double> env_flops, env_nnz;
  // A in the cluster order (for the SpMV of PCG)
  std::vector<int64_t> prow;
  std::vector<int32_t> pcol;
  std::vector<int64_t> pval_src;
  // device
  int device = -1;
  bool consts_ready = false;
  DevArena persist, descs;
  PinnedStage stage;  // host side of every descriptor upload of a factorization
  DevBuf scratch[2];
  DevBuf d_vals, d_asm_row, d_asm_off, d_prow, d_pcol, d_pval, d_pval_src, d_perm;
  DevBuf d_vec, d_tmp, d_save, d_bin, d_bout;
  DevBuf d_piv64;  // FP64 copies of the pivot blocks of FP32 factors (scratch)
  DevBuf d_rand;   // sketches, products and state of the randomized compression (scratch)
  DevBuf d_interp; // Gram matrices, R rows and pivot orders of the interpolative variants (scratch)
  // host scratch reused across steps and factorizations
  VecPool<int32_t> pool32;
  // Per step, the structure of the elimination's Schur update (which target
  // blocks, which contributions, in which order): fixed by the analysis, so
  // built at the first factorization and reused by every later one.
  struct SchurPlan {
    bool built = false;
    std::vector<int32_t> a, b, eab, eba;      // target block (a, b), a's edge to b and b's edge to a (-1: a == b)
    std::vector<int32_t> cptr, csep, cea, ceb;  // its contributions: separator, its edges to a and to b
  };
  std::vector<SchurPlan> splan;
  // Per step, the block copies of the merge (Sec. 2.7): for every remaining
  // cluster a, its own block and each neighbour b, with b's edge in a's row
  // (-1: a itself) and the edge of the parents (P, Q) in the next layout (-1:
  // P == Q; -2: not adjacent there, nothing to copy); fixed by the analysis.
  struct MergePlan {
    bool built = false;
    std::vector<int32_t> ptr, b, src, tgt;  // per entry of rems: ptr[i] .. ptr[i + 1]
  };
  std::vector<MergePlan> mplan;
  VecPool<int64_t> pool64;
  VecPool<std::pair<int32_t, int64_t>> poolpair;
  VecPool<ApplyItem> poolitem;
  std::vector<int64_t> gb_head, gb_byslot;  // the scatter grouping's counting sort
  DevBuf d_rowptr, d_colind;  // original CSR pattern (gradient on A's pattern)
  int fprec = -1;
  bool factored = false;
  std::vector<ApplyStep<double>> apply64;
  std::vector<ApplyStep<float>> apply32;
  int64_t tmp_len = 0, save_len = 0;
  spand_stats st{};
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};
  std::vector<std::vector<int32_t>> sizes_before, sizes_after;
  cudaStream_t aux[kAuxStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kAuxStreams] = {};
  cudaStream_t qs = nullptr;                         // Q_pc formation, one colour behind the QR kernels
  cudaEvent_t ev_q = nullptr, ev_qdone = nullptr;
  KProf prof;
  // the preconditioner apply program (phases of every step, on the device);
  // one cooperative launch of k_apply runs it
  const void* aprog = nullptr;
  int n_aprog = 0;
  int apply_grid = 0;
  int apply_per_sm_max = 1;  // occupancy limit of the apply kernel for this program
  int apply_ctas = 0;        // CTAs per SM of the apply: 0 = not chosen yet (autotuned at the first apply)
  size_t apply_smem = 0;
  DevBuf d_bar;  // [0] grid-barrier arrival counter, [1] barrier-timeout flag
  unsigned apply_spin_limit = kBarrierSpins;  // polls per grid-barrier wait of the apply
  unsigned apply_bias = 0;                    // 1: failure-path test, no barrier completes
  ~spand_handle_s() {
    for (auto& a : aux)
      if (a) cudaStreamDestroy(a);
    if (qs) cudaStreamDestroy(qs);
    if (ev_q) cudaEventDestroy(ev_q);
    if (ev_qdone) cudaEventDestroy(ev_qdone);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto& e : ev_join)
      if (e) cudaEventDestroy(e);
  }
};

namespace spand {

// ---------------------------------------------------------------- layouts

template <typename T>
struct Layout {
  std::vector<T*> row;
  std::vector<int32_t> ld, W;
  std::vector<int32_t> nptr, nidx, noff;  // neighbour lists with column offsets
  int32_t edge_of(int i, int q) const {  // index of q in i's neighbour list, or -1
    const int32_t* b = nidx.data() + nptr[i];
    const int32_t* e = nidx.data() + nptr[i + 1];
    const int32_t* it = std::lower_bound(b, e, q);
    return (it == e || *it != q) ? -1 : nptr[i] + (int32_t)(it - b);
  }
  int32_t off_of(int i, int q) const {
    if (q == i) return 0;
    const int32_t* b = nidx.data() + nptr[i];
    const int32_t* e = nidx.data() + nptr[i + 1];
    const int32_t* it = std::lower_bound(b, e, q);
    if (it == e || *it != q) return -1;
    return noff[nptr[i] + (it - b)];
  }
  int32_t first_upper(int i) const {  // column where the blocks of neighbours q > i start
    for (int32_t e = nptr[i]; e < nptr[i + 1]; ++e)
      if (nidx[e] > i) return noff[e];
    return W[i];
  }
};

// Row layout of step t: eliminated clusters keep their pre-elimination
// neighbours (cluster graph before the step), the others the graph after the
// step's fill.  Separator rows go to the persistent arena (they are factor
// data), the others to the step's scratch buffer.
template <typename T>
static Layout<T> make_layout(spand_handle h, int t, const std::vector<int32_t>& sz, cudaStream_t s) {
  const StepStruct& st = h->tree.steps[t - 1];
  Layout<T> lay;
  const int n = st.n;
  lay.row.assign(n, nullptr);
  lay.ld.resize(n);
  lay.W.resize(n);
  lay.nptr.assign(1, 0);
  for (int i = 0; i < n; ++i) {
    const int32_t* b = st.elim[i] ? &st.adj_idx[st.adj_ptr[i]] : &st.adjf_idx[st.adjf_ptr[i]];
    const int32_t* e = st.elim[i] ? &st.adj_idx[st.adj_ptr[i + 1]] : &st.adjf_idx[st.adjf_ptr[i + 1]];
    int32_t w = sz[i];
    for (const int32_t* q = b; q < e; ++q) {
      lay.nidx.push_back(*q);
      lay.noff.push_back(w);
      w += sz[*q];
    }
    lay.nptr.push_back((int32_t)lay.nidx.size());
    lay.W[i] = w;
    lay.ld[i] = row_ld(sz[i]);
  }
  size_t pers = 0, scr = 0;
  for (int i = 0; i < n; ++i) {
    size_t b = align256((size_t)lay.ld[i] * std::max(lay.W[i], 1) * sizeof(T));
    (st.elim[i] ? pers : scr) += b;
  }
  char* pbase = pers ? (char*)h->persist.alloc(pers) : nullptr;
  char* sbase = scr ? (char*)h->scratch[t & 1].ensure(scr) : nullptr;
  size_t po = 0, so = 0;
  for (int i = 0; i < n; ++i) {
    size_t b = align256((size_t)lay.ld[i] * std::max(lay.W[i], 1) * sizeof(T));
    if (st.elim[i]) { lay.row[i] = (T*)(pbase + po); po += b; }
    else { lay.row[i] = (T*)(sbase + so); so += b; }
  }
  if (pers) CK(cudaMemsetAsync(pbase, 0, pers, s));
  if (scr) CK(cudaMemsetAsync(sbase, 0, scr, s));
  return lay;
}

static void ensure_streams(spand_handle h) {
  if (h->ev_fork) return;
  for (auto& a : h->aux) CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->qs, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_q, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_qdone, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  for (auto& e : h->ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

template <typename T>
static void* upload(spand_handle h, const Packer& pk, cudaStream_t s) {
  if (pk.empty()) return nullptr;
  void* d = h->descs.alloc(pk.size);
  void* src = h->stage.take(pk.size);
  pk.write(src);
  CK(cudaMemcpyAsync(d, src, pk.size, cudaMemcpyHostToDevice, s));
  return d;
}

template <typename X>
static X* at(void* base, size_t off) { return reinterpret_cast<X*>((char*)base + off); }

// Launch with programmatic stream serialization: the kernel may be scheduled
// before its predecessor on the stream completes; the kernel itself waits
// for that completion (griddepcontrol.wait) before touching its data.
template <typename... P, typename... A>
static void launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CK(cudaLaunchKernelEx(&cfg, kern, args...));
}

// Tiled upper Cholesky of a batch of diagonal blocks (right-looking over
// B x B tiles; dinv and bw of the rows in B-tiles).  The phases of the tile
// steps are launched back to back as programmatic dependent launches.
template <typename T, int B = TB>
static void potrf_batch(spand_handle h, const std::vector<RowDesc<T>>& rows, int* d_info, cudaStream_t s,
                        const std::vector<double>* row_flops = nullptr) {
  if (rows.empty()) return;
  Packer pk;
  size_t o = pk.add(rows);
  void* d = upload<T>(h, pk, s);
  const RowDesc<T>* dr = at<const RowDesc<T>>(d, o);
  int nmax = 0;
  for (auto& r : rows) nmax = std::max(nmax, r.n);
  const int nt = (nmax + B - 1) / B;
  const size_t sm1 = 2 * sizeof(SqTileB<T, B>), sm2 = 2 * sizeof(SqTileB<T, B>);
  ensure_smem((const void*)k_potrf_diag<T, B>, sm1);
  ensure_smem((const void*)k_potrf_trsm<T, B>, sm2);
  constexpr int nth = TileGeom<B>::NTH;
  const int nb = (int)rows.size();
  double fl = 0, by = 0;
  for (size_t i = 0; i < rows.size(); ++i) {
    const RowDesc<T>& r = rows[i];
    fl += row_flops ? (*row_flops)[i] : (double)r.n * r.n * r.n / 3;
    by += 2.0 * r.n * r.n * sizeof(T);
  }
  const int pid = h->prof.begin(F_POTRF, s);
  int64_t nl = 0;
  for (int k = 0; k < nt; ++k) {
    nl += (nt - k - 1 > 0) ? 3 : 1;
    launch_pdl(k_potrf_diag<T, B>, dim3(nb), dim3(nth), sm1, s, dr, k, d_info);
    const int m = nt - k - 1;
    if (m > 0) {
      launch_pdl(k_potrf_trsm<T, B>, dim3(m, nb), dim3(nth), sm2, s, dr, k);
      launch_pdl(k_potrf_update<T, B>, dim3(m * (m + 1) / 2, nb), dim3(nth), (size_t)0, s, dr, k);
    }
  }
  h->prof.launches += nl;
  h->prof.end(pid, s, fl, by, nl);
}

// U_kk^{-T} of every 64 x 64 diagonal tile of a batch of factored pivot
// blocks (rows: R = U, dinv = destination), for the block-row solves.
template <typename T>
static void inv_diag_batch(spand_handle h, const std::vector<RowDesc<T>>& rows, cudaStream_t s) {
  if (rows.empty()) return;
  Packer pk;
  size_t o = pk.add(rows);
  void* d = upload<T>(h, pk, s);
  int nmax = 0;
  for (auto& r : rows) nmax = std::max(nmax, r.n);
  const int nt = (nmax + TB - 1) / TB;
  const size_t sm = 2 * sizeof(SqTile<T>);
  ensure_smem((const void*)k_inv_diag<T>, sm);
  const size_t nb = rows.size();
  for (size_t b0 = 0; b0 < nb; b0 += 65535) {
    const unsigned cnt = (unsigned)std::min<size_t>(nb - b0, 65535);
    k_inv_diag<T><<<dim3(nt, cnt), INV_NT, sm, s>>>(at<const RowDesc<T>>(d, o) + b0);
    CKLAUNCH();
    ++h->prof.launches;
  }
}

// Cholesky of a batch of pivot blocks in FP64 (Sec. 2.4, 2.5), on 32 x 32
// tiles: FP64 factors are factored in place; FP32 factors (the mixed forms)
// are widened into an FP64 scratch copy, factored there, and U is rounded
// back to FP32.  Then the inverses of U's 64 x 64 diagonal tiles (rows'
// dinv, in the factor's precision) for the block-row solves.
template <typename T>
static void pivot_chol(spand_handle h, const std::vector<RowDesc<T>>& rows, int* d_info, cudaStream_t s,
                       const std::vector<double>* row_flops = nullptr) {
  if (rows.empty()) return;
  const bool wide = !std::is_same<T, double>::value;
  size_t tot = 0;
  for (auto& r : rows)
    tot += (wide ? ((size_t)r.n * r.n + 31) / 32 * 32 : 0) + (size_t)((r.n + TB2 - 1) / TB2) * TB2 * TB2;
  double* base = (double*)h->d_piv64.ensure(std::max<size_t>(tot, 1) * sizeof(double));
  std::vector<RowDesc<double>> r64;
  std::vector<PivotCopy> cps;
  r64.reserve(rows.size());
  // banded blocks (step-1 pivots with a narrow band) go to the banded kernel,
  // on their own storage (no FP64 copy); the tiled batch skips them (n = 0
  // keeps the batch indices, which the failure flag reports)
  std::vector<BandTask<T>> bands;
  int bmax = 0;
  size_t o = 0;
  for (size_t i = 0; i < rows.size(); ++i) {
    const RowDesc<T>& r = rows[i];
    if (r.band > 0 && r.band <= BAND_MAX && r.band + 1 < r.n) {
      bands.push_back({r.R, r.n, r.ld, r.band, (int32_t)i});
      bmax = std::max(bmax, r.band);
      r64.push_back({nullptr, 0, 1, nullptr, 0, 0});
      continue;
    }
    double* W = nullptr;
    if (wide) {
      W = base + o;
      o += ((size_t)r.n * r.n + 31) / 32 * 32;
      cps.push_back({(float*)r.R, W, r.n, r.ld});
    }
    double* D = base + o;
    o += (size_t)((r.n + TB2 - 1) / TB2) * TB2 * TB2;
    if (wide) r64.push_back({W, r.n, r.n, D, r.bw2, 0});
    else r64.push_back({(double*)r.R, r.n, r.ld, D, r.bw2, 0});
  }
  bool dense_left = false;
  for (const auto& r : r64) dense_left = dense_left || r.n > 0;
  const PivotCopy* dc = nullptr;
  if (wide && !cps.empty()) {
    Packer pk;
    const size_t oc = pk.add(cps);
    void* d = upload<T>(h, pk, s);
    dc = at<const PivotCopy>(d, oc);
    for (size_t b0 = 0; b0 < cps.size(); b0 += 65535) {
      const unsigned cnt = (unsigned)std::min<size_t>(cps.size() - b0, 65535);
      k_widen_pivot<<<dim3(8, cnt), 256, 0, s>>>(dc + b0);
      CKLAUNCH();
      ++h->prof.launches;
    }
  }
  if (!bands.empty()) {
    Packer pk;
    const size_t ob = pk.add(bands);
    void* d = upload<T>(h, pk, s);
    const size_t sm = band_smem(bmax);
    ensure_smem((const void*)k_potrf_band<T>, sm);
    const int pid = h->prof.begin(F_POTRF, s);
    for (size_t b0 = 0; b0 < bands.size(); b0 += 65535) {
      const unsigned cnt = (unsigned)std::min<size_t>(bands.size() - b0, 65535);
      launch_pdl(k_potrf_band<T>, dim3(cnt), dim3(BAND_NT), sm, s, at<const BandTask<T>>(d, ob) + b0, d_info);
      ++h->prof.launches;
    }
    double fl = 0, by = 0;
    for (const BandTask<T>& b : bands) {
      fl += row_flops ? (*row_flops)[b.entry] : (double)b.n * b.band * b.band;
      by += 2.0 * b.n * (b.band + 1) * sizeof(T);
    }
    h->prof.end(pid, s, fl, by, (int64_t)((bands.size() + 65534) / 65535));
  }
  if (dense_left) potrf_batch<double, TB2>(h, r64, d_info, s, row_flops);
  if (wide && !cps.empty()) {
    for (size_t b0 = 0; b0 < cps.size(); b0 += 65535) {
      const unsigned cnt = (unsigned)std::min<size_t>(cps.size() - b0, 65535);
      k_narrow_pivot<<<dim3(8, cnt), 256, 0, s>>>(dc + b0);
      CKLAUNCH();
      ++h->prof.launches;
    }
  }
  inv_diag_batch<T>(h, rows, s);
}

template <typename T>
static void trsm_batch(spand_handle h, const std::vector<TrsmTask<T>>& tasks, cudaStream_t s,
                       const std::vector<double>* task_flops = nullptr) {
  if (tasks.empty()) return;
  Packer pk;
  size_t o = pk.add(tasks);
  void* d = upload<T>(h, pk, s);
  const size_t sm = 2 * sizeof(SqTile<T>) + sizeof(TileSmem<T>);
  ensure_smem((const void*)k_trsm_cols<T>, sm);
  double fl = 0, by = 0;
  for (size_t i = 0; i < tasks.size(); ++i) {
    const TrsmTask<T>& t = tasks[i];
    const double nn = t.n - (t.i_start / TB) * TB;
    fl += task_flops ? (*task_flops)[i] : nn * nn * t.nc;
    by += (nn * nn / 2 + 2.0 * nn * t.nc) * sizeof(T);
  }
  const int pid = h->prof.begin(F_TRSM, s);
  k_trsm_cols<T><<<(unsigned)tasks.size(), NT, sm, s>>>(at<const TrsmTask<T>>(d, o));
  CKLAUNCH();
  h->prof.launches += 1;
  h->prof.end(pid, s, fl, by, 1);
}

// Panels of at most 64 columns [c0, c1) of a block row: B <- U^{-T} B.
// fl (optional): receives each task's algorithmic flops, 2 nnz(U) per column
// (nnzU: nonzeros of U's upper triangle, n (n + 1) / 2 when dense).
template <typename T>
static void add_panels(std::vector<TrsmTask<T>>& out, T* R, const T* dinv, int n, int ld, int c0, int c1,
                       int bw = 0, std::vector<double>* fl = nullptr, double nnzU = -1) {
  if (n <= 0) return;
  if (nnzU < 0) nnzU = (double)n * (n + 1) / 2;
  for (int c = c0; c < c1; c += TB) {
    TrsmTask<T> t;
    t.U = R;
    t.dinv = dinv;
    t.B = R + (size_t)c * ld;
    t.n = n;
    t.ldu = ld;
    t.ldb = ld;
    t.nc = std::min(c + TB, c1) - c;
    t.i_start = 0;
    t.bw = bw;
    out.push_back(t);
    if (fl) fl->push_back(2.0 * nnzU * t.nc);
  }
}

// Y = U^{-T} (lower): the same solve on identity panels (Y must hold I).
template <typename T>
static void add_inverse(std::vector<TrsmTask<T>>& out, const T* U, const T* dinv, int n, int ldu, T* Y,
                        int bw = 0, std::vector<double>* fl = nullptr) {
  for (int c = 0; c < n; c += TB) {
    TrsmTask<T> t;
    t.U = U;
    t.dinv = dinv;
    t.B = Y + (size_t)c * n;
    t.n = n;
    t.ldu = ldu;
    t.ldb = n;
    t.nc = std::min(c + TB, n) - c;
    t.i_start = c;
    t.bw = bw;
    out.push_back(t);
    if (fl) {  // rows [c, n) of a lower-triangular panel: ~ (n - c)^2 per column
      const double nn = n - c;
      fl->push_back(nn * nn * t.nc);
    }
  }
}

template <typename T>
static void set_identity(spand_handle h, const std::vector<RowDesc<T>>& rows, cudaStream_t s);

// Storage for the inverses of the diagonal 64x64 tiles of an n x n pivot block.
template <typename T>
static T* alloc_dinv(spand_handle h, int n) {
  const size_t nt = (size_t)(n + TB - 1) / TB;
  return (T*)h->descs.alloc(std::max<size_t>(nt, 1) * TB * TB * sizeof(T));
}

template <typename T>
static void copy_batch(spand_handle h, const std::vector<CopyTask<T>>& tasks_in, cudaStream_t s) {
  if (tasks_in.empty()) return;
  // tasks without tiles are left out (the kernel's search assumes none)
  const std::vector<CopyTask<T>>* tp = &tasks_in;
  std::vector<CopyTask<T>> kept;
  for (const CopyTask<T>& c : tasks_in)
    if (c.rows <= 0 || c.cols <= 0) {
      for (const CopyTask<T>& k : tasks_in)
        if (k.rows > 0 && k.cols > 0) kept.push_back(k);
      tp = &kept;
      break;
    }
  const std::vector<CopyTask<T>>& tasks = *tp;
  if (tasks.empty()) return;
  // prefix sums of the tasks' 32 x 32 tile counts, and the task of every 32nd tile
  std::vector<int32_t> tptr = h->pool32.take(), cidx = h->pool32.take();
  tptr.resize(tasks.size() + 1);
  int64_t ntile = 0;
  for (size_t i = 0; i < tasks.size(); ++i) {
    tptr[i] = (int32_t)std::min<int64_t>(ntile, INT32_MAX);
    ntile += (int64_t)((tasks[i].rows + 31) / 32) * ((tasks[i].cols + 31) / 32);
  }
  if (ntile > INT32_MAX - 64) {
    h->pool32.give(std::move(tptr));
    h->pool32.give(std::move(cidx));
    throw Fail{SPAND_ERR_INVALID_ARG, "block copy batch too large"};
  }
  tptr[tasks.size()] = (int32_t)ntile;
  cidx.resize((size_t)((ntile + 31) / 32));
  for (size_t c = 0, i = 0; c < cidx.size(); ++c) {
    const int64_t g = (int64_t)c * 32;
    while (tptr[i + 1] <= g) ++i;
    cidx[c] = (int32_t)i;
  }
  Packer pk;
  size_t ot = pk.add(tasks), op = pk.add(tptr), oc = pk.add(cidx);
  void* d = upload<T>(h, pk, s);
  h->pool32.give(std::move(tptr));  // copied to pinned staging by upload
  h->pool32.give(std::move(cidx));
  double by = 0;
  for (auto& t : tasks) by += 2.0 * t.rows * t.cols * sizeof(T);
  const int pid = h->prof.begin(F_COPY, s);
  const unsigned nb = (unsigned)((ntile + CP_WARPS - 1) / CP_WARPS);
  k_copy<T><<<nb, 32 * CP_WARPS, 0, s>>>(at<const int32_t>(d, op), at<const int32_t>(d, oc), (int)tasks.size(),
                                          (int32_t)ntile, at<const CopyTask<T>>(d, ot));
  CKLAUNCH();
  h->prof.launches += 1;
  h->prof.end(pid, s, 0.0, by, 1);
}

template <typename T>
static void set_identity(spand_handle h, const std::vector<RowDesc<T>>& rows, cudaStream_t s) {
  if (rows.empty()) return;
  Packer pk;
  size_t o = pk.add(rows);
  void* d = upload<T>(h, pk, s);
  k_set_identity<T><<<dim3(8, (unsigned)rows.size()), 256, 0, s>>>(at<const RowDesc<T>>(d, o), (int)rows.size());
  CKLAUNCH();
  h->prof.launches += 1;
}

// Phase boundaries of every step (5 events per step, read once at the end of
// the factorization, so that no step waits for its own timing).
struct StepTimer {
  std::vector<cudaEvent_t> ev;
  explicit StepTimer(int nsteps) : ev(5 * (size_t)(nsteps + 1), nullptr) {
    for (auto& e : ev) CK(cudaEventCreate(&e));
  }
  cudaEvent_t at(int t, int k) const { return ev[5 * (size_t)t + k]; }
  ~StepTimer() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Register-resident sparsification (FP32 factors): 512 threads per CTA, 64
// rows per lane, lane groups of G = 1..8 lanes per column, so an interface
// of np <= 512 rows and m columns takes ceil(m / (512 / G)) CTAs (<= 16).
constexpr int kCqrThreads = 512;
constexpr int kCqrRows = 64;
constexpr int kCqrMaxCluster = 16;

template <typename T>
static const void* cpqr_reg_kernel(int G) {
  if constexpr (sizeof(T) != 4) {
    return nullptr;
  } else {
    switch (G) {
      case 1: return (const void*)k_cpqr_reg<float, kCqrThreads, 1, kCqrRows>;
      case 2: return (const void*)k_cpqr_reg<float, kCqrThreads, 2, kCqrRows>;
      case 4: return (const void*)k_cpqr_reg<float, kCqrThreads, 4, kCqrRows>;
      case 8: return (const void*)k_cpqr_reg<float, kCqrThreads, 8, kCqrRows>;
      default: return nullptr;
    }
  }
}

template <typename T>
static size_t cpqr_reg_smem(int G, int nnb, int np, int cols_per, int C) {
  switch (G) {
    case 1: return cqr_smem<T, kCqrThreads, 1, kCqrRows>(nnb, np, cols_per, C);
    case 2: return cqr_smem<T, kCqrThreads, 2, kCqrRows>(nnb, np, cols_per, C);
    case 4: return cqr_smem<T, kCqrThreads, 4, kCqrRows>(nnb, np, cols_per, C);
    default: return cqr_smem<T, kCqrThreads, 8, kCqrRows>(nnb, np, cols_per, C);
  }
}

static std::mutex g_cqr_mutex;  // guards the cached cluster capacities

// How many clusters of C register-resident CTAs (lane groups of G) can be
// resident at once on this device (0 when the shape cannot launch).
template <typename T>
static int cpqr_reg_capacity(int G, int C) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_cqr_mutex);
  static std::map<std::tuple<int, int, int>, int> cached;
  auto it = cached.find({dev, G, C});
  if (it != cached.end()) return it->second;
  const void* fn = cpqr_reg_kernel<T>(G);
  int n = 0;
  if (fn) {
    const size_t smem = 227 * 1024;  // one CTA per SM either way (registers)
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
        (C <= 8 || cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)C, 1, 1);
      cfg.blockDim = dim3((unsigned)kCqrThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();  // a refused query only means "not this shape"
  }
  cached[{dev, G, C}] = n;
  return n;
}

// The sparsification kernel for a launch group: chunk in shared memory or
// not, 256 or 512 threads per CTA.
template <typename T>
static const void* cpqr_kernel(bool res, int nt, int lg = 1) {
  if (nt == 512 && lg == 4)
    return res ? (const void*)k_cpqr_cluster<T, true, 512, 4> : (const void*)k_cpqr_cluster<T, false, 512, 4>;
  if (nt == 512 && lg == 2)
    return res ? (const void*)k_cpqr_cluster<T, true, 512, 2> : (const void*)k_cpqr_cluster<T, false, 512, 2>;
  if (res) return nt == 512 ? (const void*)k_cpqr_cluster<T, true, 512> : (const void*)k_cpqr_cluster<T, true, 256>;
  return nt == 512 ? (const void*)k_cpqr_cluster<T, false, 512> : (const void*)k_cpqr_cluster<T, false, 256>;
}

// Randomized compression (SPAND_RANDOMIZED) of the interfaces of one step,
// colour by colour (the kernels and the method are described in
// sparsify_rand.cuh).  The column-pivoted QR of each sketch runs on the
// chunked QR kernel as a task of its own (the sketch Y as its coupling
// block, no write-back); between rounds the host reads which interfaces
// still need a wider sketch.  Returns each task's final sketch width.
template <typename T>
static std::vector<int> sparsify_randomized(spand_handle h, int t, const std::vector<CpqrTask<T>>& tasks,
                                            const std::vector<int>& tcolour, int ncol,
                                            const std::vector<CpqrNbr<T>>& nbrs, int32_t* d_cur, double eps,
                                            cudaStream_t s) {
  const size_t ntk = tasks.size();
  std::vector<int> ell_final(ntk, 0);
  if (ntk == 0) return ell_final;
  struct Off { size_t om, y, w, tcol, res, gw; };
  std::vector<Off> off(ntk);
  size_t bytes = 0;
  for (size_t i = 0; i < ntk; ++i) {
    const size_t np = (size_t)std::max(tasks[i].np, 1), mm = (size_t)std::max(tasks[i].m_max, 1);
    const size_t Lp = (size_t)cq_ld<T>((int)np), cap = std::min(np, mm);
    off[i].om = bytes; bytes += align256(mm * np * sizeof(T));
    off[i].y = bytes; bytes += align256(np * np * sizeof(T));
    off[i].w = bytes; bytes += align256(np * mm * sizeof(T));
    off[i].tcol = bytes; bytes += align256(mm * sizeof(int32_t));
    off[i].res = bytes; bytes += align256((np + 2) * sizeof(unsigned long long));
    off[i].gw = bytes; bytes += align256(Lp * (cap + 16) * sizeof(T));
  }
  char* base = (char*)h->d_rand.ensure(bytes);
  Packer pkn;
  const size_t onb = pkn.add(nbrs);
  const CpqrNbr<T>* d_nbrs = at<const CpqrNbr<T>>(upload<T>(h, pkn, s), onb);
  const size_t CB = kCpqrChunkBudget;
  const int max_cluster = cpqr_max_cluster<T>();
  const uint64_t seed = h->opts.sketch_seed;
  int32_t* hbuf = nullptr;
  for (int c = 0; c < std::max(ncol, 1); ++c) {
    std::vector<int> ids;
    for (size_t i = 0; i < ntk; ++i)
      if (tcolour[i] == c) ids.push_back((int)i);
    const int nc = (int)ids.size();
    if (nc == 0) continue;
    std::vector<RandTask<T>> rt(nc);
    std::vector<CpqrTask<T>> vt(nc);
    std::vector<CpqrNbr<T>> vn(nc);
    int npmax = 1, mmax = 1;
    for (int k = 0; k < nc; ++k) {
      const CpqrTask<T>& tk = tasks[ids[k]];
      const Off& o = off[ids[k]];
      RandTask<T> r{};
      r.Rp = tk.Rp;
      r.Om = (T*)(base + o.om);
      r.Y = (T*)(base + o.y);
      r.W = (T*)(base + o.w);
      r.Qc = tk.Qc;
      r.tcol = (int32_t*)(base + o.tcol);
      r.res = (unsigned long long*)(base + o.res);
      r.p = tk.p;
      r.np = tk.np;
      r.ldp = tk.ldp;
      r.nbeg = tk.nbeg;
      r.nend = tk.nend;
      r.m_max = tk.m_max;
      rt[k] = r;
      CpqrTask<T> v = tk;  // V, tau and Qc of the interface; the sketch is the coupling block
      v.Rp = r.Y;
      v.ldp = std::max(tk.np, 1);
      v.gwork = (T*)(base + o.gw);
      v.rank_out = nullptr;  // set after the upload (the rank array of the sketches)
      v.p = k;
      v.nbeg = k;
      v.nend = k + 1;
      v.m_max = std::min(tk.np, tk.m_max);
      v.nowb = 1;
      vt[k] = v;
      CpqrNbr<T> nb{};
      nb.Rq = r.Y;
      nb.q = k;
      nb.off_pq = 0;
      nb.off_qp = 0;
      nb.ldq = std::max(tk.np, 1);
      vn[k] = nb;
      npmax = std::max(npmax, tk.np);
      mmax = std::max(mmax, tk.m_max);
      if (tk.nend - tk.nbeg > 256)
        throw Fail{SPAND_ERR_INVALID_ARG, "randomized compression: an interface with more than 256 neighbours"};
    }
    // device state: [vcur | vrank | active] ints, then the task arrays
    Packer pk;
    const std::vector<int32_t> state0((size_t)3 * nc, 0);
    const size_t ostate = pk.add(state0);
    const size_t ort = pk.add(rt), ovn = pk.add(vn);
    const size_t ovt = pk.add(vt);
    void* dev = h->descs.alloc(pk.size);
    int32_t* d_vcur = at<int32_t>(dev, ostate);
    int32_t* d_vrank = d_vcur + nc;
    int32_t* d_active = d_vcur + 2 * nc;
    for (int k = 0; k < nc; ++k) vt[k].rank_out = d_vrank;  // the device copy's rank array
    {
      void* src = h->stage.take(pk.size);
      pk.write(src);
      CK(cudaMemcpyAsync(dev, src, pk.size, cudaMemcpyHostToDevice, s));
    }
    RandTask<T>* d_rt = at<RandTask<T>>(dev, ort);
    CpqrTask<T>* d_vt = at<CpqrTask<T>>(dev, ovt);
    const CpqrNbr<T>* d_vn = at<const CpqrNbr<T>>(dev, ovn);
    k_rand_init<T><<<nc, 256, 0, s>>>(d_rt, d_nbrs, d_cur, d_vcur);
    CKLAUNCH();
    std::vector<int> ub(nc), act(nc, 1), prev(nc, 0);
    for (int k = 0; k < nc; ++k) ub[k] = std::min(RD_ELL0, std::max(0, std::min(rt[k].np, rt[k].m_max)));
    int64_t nl = 1;
    for (;;) {
      std::vector<int32_t> alist;
      int maxub = 1, maxnew = 1;
      for (int k = 0; k < nc; ++k)
        if (act[k]) {
          alist.push_back(k);
          maxub = std::max(maxub, ub[k]);
          maxnew = std::max(maxnew, ub[k] - prev[k]);
        }
      if (alist.empty()) break;
      k_rand_omega<T><<<dim3(32, nc), 256, 0, s>>>(d_rt, seed, t);
      CKLAUNCH();
      const int tiles = ((npmax + 31) / 32) * ((maxnew + 31) / 32);
      k_rand_sketch<T><<<dim3(tiles, nc), 256, 0, s>>>(d_rt);
      CKLAUNCH();
      // the QR of every active sketch, grouped by launch shape
      std::map<std::tuple<int, int, int>, std::vector<int32_t>> groups;  // (C, resident, threads) -> tasks
      std::map<std::tuple<int, int, int>, size_t> gsmem;
      for (int k : alist) {
        // sized for the task's column bound vt.m_max, from which the kernel
        // lays out its shared memory (not for this round's width ub[k] <= it)
        const int np = std::max(rt[k].np, 1), cols = std::max(vt[k].m_max, 1);
        const size_t Lp = (size_t)cq_ld<T>(np);
        auto res_smem = [&](int cc) {
          const int cp = (cols + cc - 1) / cc;
          return cq_fixed_smem<T>(1, np, cp, cc) + Lp * cp * sizeof(T);
        };
        int C = max_cluster;
        for (int cc = 1; cc <= max_cluster; cc *= 2)
          if (res_smem(cc) <= CB) { C = cc; break; }
        while (C < max_cluster && (cols + C - 1) / C > 2 * CQ_MAXNT) C *= 2;
        const bool resident = res_smem(C) <= CB;
        const int cp = (cols + C - 1) / C;
        const int nth = cp > CQ_CPT * 256 ? 512 : 256;
        const auto key = std::make_tuple(C, resident ? 1 : 0, nth);
        groups[key].push_back(k);
        const size_t need = resident ? res_smem(C) : cq_fixed_smem<T>(1, np, cp, C);
        gsmem[key] = std::max(gsmem[key], need);
      }
      Packer pkl;
      std::vector<size_t> lo;
      for (auto& kv : groups) lo.push_back(pkl.add(kv.second));
      const size_t oal = pkl.add(alist);
      void* dl = upload<T>(h, pkl, s);
      size_t gi = 0;
      for (auto& kv : groups) {
        const int C = std::get<0>(kv.first), res = std::get<1>(kv.first), nth = std::get<2>(kv.first);
        const void* fn = cpqr_kernel<T>(res != 0, nth);
        const size_t smem = gsmem[kv.first];
        ensure_smem(fn, smem);
        if (C > 8) ensure_nonportable_cluster(fn);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(kv.second.size() * C), 1, 1);
        cfg.blockDim = dim3((unsigned)nth, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const CpqrTask<T>* a0 = d_vt;
        const int32_t* a1 = at<const int32_t>(dl, lo[gi]);
        const CpqrNbr<T>* a2 = d_vn;
        T a4 = T(0);  // no truncation: the rank comes from step 5
        void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&d_vcur, (void*)&a4};
        CK(cudaLaunchKernelExC(&cfg, fn, args));
        ++gi;
        ++nl;
      }
      {  // the bases Q = H_0 ... H_{ell-1} [I; 0]
        constexpr int NTQ = 256, NWQ = NTQ / 32;
        int kmx = 1;
        size_t need = 0;
        for (int k : alist) {
          const int km = std::min(rt[k].np, ub[k]);
          kmx = std::max(kmx, km);
          need = std::max(need, align256((size_t)km * sizeof(T)) + (size_t)rt[k].np * km * sizeof(T));
        }
        const size_t qsm = std::min(need + 256, (size_t)227 * 1024);
        const int nb = std::max(1, (kmx + 2 * NWQ - 1) / (2 * NWQ));
        const void* fq = (const void*)k_form_q<T, NTQ>;
        ensure_smem(fq, qsm);
        const CpqrTask<T>* q0 = d_vt;
        const int32_t* q1 = at<const int32_t>(dl, oal);
        const int q3 = nb, q4 = (int)(qsm / sizeof(T));
        void* qargs[] = {(void*)&q0, (void*)&q1, (void*)&d_vcur, (void*)&q3, (void*)&q4};
        CK(cudaLaunchKernel(fq, dim3((unsigned)(alist.size() * nb)), dim3(NTQ), qargs, qsm, s));
        ++nl;
      }
      k_rand_project<T><<<dim3((unsigned)((mmax + 31) / 32), nc), 256, 0, s>>>(d_rt);
      CKLAUNCH();
      k_rand_decide<T><<<(nc + 127) / 128, 128, 0, s>>>(d_rt, nc, eps, d_vcur, d_vt, d_active);
      CKLAUNCH();
      nl += 5;
      // which sketches must grow, and to what width
      if (!hbuf) hbuf = (int32_t*)h->stage.take((size_t)2 * ntk * sizeof(int32_t) + 256);
      CK(cudaMemcpyAsync(hbuf, d_vcur, (size_t)nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hbuf + nc, d_active, (size_t)nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int k : alist) {
        ell_final[ids[k]] = ub[k];
        act[k] = hbuf[nc + k];
        if (act[k]) {
          prev[k] = ub[k];
          ub[k] = hbuf[k];
        }
      }
    }
    k_rand_writeback<T><<<dim3((unsigned)std::min(32, (mmax + npmax + 63) / 64), nc), 256, 0, s>>>(d_rt, d_nbrs,
                                                                                                  d_cur);
    CKLAUNCH();
    h->prof.launches += nl + 1;
  }
  return ell_final;
}

// Result of the interpolative sparsification of one interface.
template <typename T>
struct InterpOut {
  int p = -1, r = 0, nf = 0, ldf = 0;
  std::vector<int32_t> perm;  // c (pivot order), then f (increasing)
  const T* F = nullptr;       // [U_f | X_fc] after the elimination of f (ld ldf)
  const T* XT = nullptr;      // T_cf (r x nf, ld r)
  const T* Yf = nullptr;      // U_f^{-T} (nf x nf)
};

// Interpolative sparsification (SPAND_INS / SPAND_IN) of the interfaces of
// one step, colour by colour (the method and its kernels are described in
// sparsify_interp.cuh).  Per colour: the Gram matrices, their truncated
// pivoted Cholesky with T_cf, and A_pp[perm, perm]; the host then reads the
// ranks and pivot orders (one synchronisation per colour: every later launch
// is shaped by them), forms C_cf and C_ff, gathers the kept blocks, and
// eliminates f with the pivot Cholesky / block-row solve / Schur kernels of
// the elimination.  hsz: the current cluster sizes (updated); d_finfo: one
// non-positive-pivot flag per colour; fcls[c]: the interface of each entry of
// colour c's pivot batch.
template <typename T>
static std::vector<InterpOut<T>> sparsify_interp(spand_handle h, const std::vector<CpqrTask<T>>& tasks,
                                                 const std::vector<int>& tcolour, int ncol,
                                                 const std::vector<CpqrNbr<T>>& nbrs, std::vector<int32_t>& hsz,
                                                 int32_t* d_cur, int* d_finfo, std::vector<std::vector<int>>& fcls,
                                                 double eps, cudaStream_t s) {
  const size_t ntk = tasks.size();
  std::vector<InterpOut<T>> out(ntk);
  fcls.assign(std::max(ncol, 1), {});
  if (ntk == 0) return out;
  // scratch: per task G, Rw, P (np^2 doubles each), the coupling copies
  // (2 np m_max), the column map (m_max); perms and ranks contiguous per colour
  struct Off { size_t g, rw, p, cp, tcol; int64_t perm; };
  std::vector<Off> off(ntk);
  size_t bytes = 0;
  int64_t nperm = 0;
  std::vector<std::vector<int>> ids(std::max(ncol, 1));
  for (size_t i = 0; i < ntk; ++i) ids[std::max(tcolour[i], 0)].push_back((int)i);
  for (const auto& col : ids)
    for (int i : col) {
      const size_t np = (size_t)std::max(tasks[i].np, 1), mm = (size_t)std::max(tasks[i].m_max, 1);
      off[i].g = bytes; bytes += align256(np * np * sizeof(double));
      off[i].rw = bytes; bytes += align256(np * np * sizeof(double));
      off[i].p = bytes; bytes += align256(np * np * sizeof(double));
      off[i].cp = bytes; bytes += align256(2 * np * mm * sizeof(T));
      off[i].tcol = bytes; bytes += align256(mm * sizeof(int32_t));
      off[i].perm = nperm;
      nperm += tasks[i].np;
    }
  const size_t operm = bytes;
  bytes += align256((size_t)std::max<int64_t>(nperm, 1) * sizeof(int32_t));
  const size_t orank = bytes;
  bytes += align256(ntk * sizeof(int32_t));
  char* base = (char*)h->d_interp.ensure(bytes);
  int32_t* d_perm = (int32_t*)(base + operm);
  int32_t* d_rank = (int32_t*)(base + orank);
  Packer pkn;
  const size_t onb = pkn.add(nbrs);
  const CpqrNbr<T>* d_nbrs = at<const CpqrNbr<T>>(upload<T>(h, pkn, s), onb);
  int32_t* hbuf = (int32_t*)h->stage.take((size_t)(nperm + (int64_t)ntk) * sizeof(int32_t) + 256);
  int64_t rank_slot = 0;  // ranks are stored in colour order too
  for (int c = 0; c < (int)ids.size(); ++c) {
    const std::vector<int>& col = ids[c];
    const int nc = (int)col.size();
    if (nc == 0) continue;
    const int pid = h->prof.begin(F_CPQR, s);
    int64_t nl = 0;
    double fl = 0, by = 0;
    std::vector<InterpTask<T>> it(nc);
    std::vector<int32_t> tcol;
    std::vector<size_t> tcol_at(nc);
    std::vector<InterpTile> gtiles;
    int npmax = 1;
    for (int k = 0; k < nc; ++k) {
      const CpqrTask<T>& tk = tasks[col[k]];
      const Off& o = off[col[k]];
      InterpTask<T> d{};
      d.Rp = tk.Rp;
      d.G = (double*)(base + o.g);
      d.Rw = (double*)(base + o.rw);
      d.P = (double*)(base + o.p);
      d.cp = (T*)(base + o.cp);
      d.perm = d_perm + o.perm;
      d.rank = d_rank + rank_slot + k;
      d.p = tk.p;
      d.np = tk.np;
      d.ldp = tk.ldp;
      d.nbeg = tk.nbeg;
      d.nend = tk.nend;
      tcol_at[k] = tcol.size();
      for (int32_t e = tk.nbeg; e < tk.nend; ++e)
        for (int32_t jj = 0; jj < hsz[nbrs[e].q]; ++jj) tcol.push_back(nbrs[e].off_pq + jj);
      d.m = (int32_t)(tcol.size() - tcol_at[k]);
      it[k] = d;
      npmax = std::max(npmax, tk.np);
      const int nt = (tk.np + 31) / 32;
      for (int ti = 0; ti < nt; ++ti)
        for (int tj = ti; tj < nt; ++tj) gtiles.push_back({k, 32 * ti, 32 * tj});
      const double np_ = tk.np, m_ = d.m;
      fl += np_ * np_ * m_;
      by += (np_ * m_ * sizeof(T) + 3.0 * np_ * np_ * sizeof(double));
    }
    {  // the column maps first, then the tasks that point into them
      Packer pk;
      const size_t ot = pk.add(tcol);
      char* d = (char*)upload<T>(h, pk, s);
      for (int k = 0; k < nc; ++k) it[k].tcol = d ? at<const int32_t>(d, ot) + tcol_at[k] : nullptr;
    }
    Packer pk;
    const size_t oi = pk.add(it), og = pk.add(gtiles);
    void* dd = upload<T>(h, pk, s);
    const InterpTask<T>* d_it = at<const InterpTask<T>>(dd, oi);
    if (!gtiles.empty()) {
      k_interp_gram<T><<<(unsigned)gtiles.size(), 256, 0, s>>>(d_it, at<const InterpTile>(dd, og));
      CKLAUNCH();
      ++nl;
    }
    const size_t fsm = (size_t)npmax * (sizeof(double) + sizeof(int));
    ensure_smem((const void*)k_interp_factor<T>, fsm);
    k_interp_factor<T><<<nc, 256, fsm, s>>>(d_it, eps);
    CKLAUNCH();
    k_interp_gather_pp<T><<<dim3(16, nc), 256, 0, s>>>(d_it);
    CKLAUNCH();
    nl += 2;
    // ranks and pivot orders of the colour
    const int64_t p0 = off[col[0]].perm;
    int64_t pn = 0;
    for (int k = 0; k < nc; ++k) pn += tasks[col[k]].np;
    CK(cudaMemcpyAsync(hbuf, d_perm + p0, (size_t)pn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hbuf + pn, d_rank + rank_slot, (size_t)nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<DGemmTask> g12, g3;
    std::vector<DGemmTile> t12, t3;
    std::vector<RowDesc<T>> ident, diag;
    std::vector<TrsmTask<T>> tr;
    std::vector<SchurBlock<T>> sblk;
    std::vector<SchurContrib<T>> scon;
    std::vector<SchurTile> stiles;
    for (int k = 0; k < nc; ++k) {
      InterpTask<T>& d = it[k];
      InterpOut<T>& o = out[col[k]];
      const int r = hbuf[pn + k];
      if (r < 0 || r > d.np) throw Fail{SPAND_ERR_STATE, "interpolative sparsification: rank out of range"};
      const int nf = d.np - r;
      o.p = d.p;
      o.r = r;
      o.nf = nf;
      o.perm.assign(hbuf + (off[col[k]].perm - p0), hbuf + (off[col[k]].perm - p0) + d.np);
      d.r = r;
      d.nf = nf;
      d.ldf = row_ld(nf);
      o.ldf = d.ldf;
      if (nf > 0) {
        const size_t fb = (size_t)d.ldf * d.np * sizeof(T);
        T* F = (T*)h->persist.alloc(fb);
        CK(cudaMemsetAsync(F, 0, fb, s));
        d.F = F;
        o.F = F;
        if (r > 0) {
          d.XT = (T*)h->persist.alloc((size_t)r * nf * sizeof(T));
          o.XT = d.XT;
        }
        T* Yf = (T*)h->persist.alloc((size_t)nf * nf * sizeof(T));
        o.Yf = Yf;
        T* dv = alloc_dinv<T>(h, nf);
        ident.push_back({Yf, nf, nf, nullptr, 0, 0});
        diag.push_back({F, nf, d.ldf, dv, 0, 0});
        fcls[c].push_back(d.p);
        add_panels(tr, F, (const T*)dv, nf, d.ldf, nf, d.np);
        add_inverse(tr, (const T*)F, (const T*)dv, nf, d.ldf, Yf);
        if (r > 0) {
          const int np = d.np;
          double* Tt = d.G;
          const int b1 = (int)g12.size();
          g12.push_back({d.P, Tt, d.P + (size_t)r * np, np, nf, np, 0, 1, r, nf, r});           // C_cf
          g12.push_back({d.P + r, Tt, d.P + r + (size_t)r * np, np, nf, np, 0, 1, nf, nf, r});  // A_ff - A_fc T
          g3.push_back({Tt, d.P + (size_t)r * np, d.P + r + (size_t)r * np, nf, np, np, 0, 0, nf, nf, r});
          for (int i0 = 0; i0 < r; i0 += 64)
            for (int j0 = 0; j0 < nf; j0 += 64) t12.push_back({b1, i0, j0});
          for (int i0 = 0; i0 < nf; i0 += 64)
            for (int j0 = 0; j0 < nf; j0 += 64) {
              t12.push_back({b1 + 1, i0, j0});
              t3.push_back({(int32_t)g3.size() - 1, i0, j0});
            }
          // A_cc -= X_fc^T X_fc
          SchurBlock<T> bl{};
          bl.C1 = d.Rp;
          bl.C2 = nullptr;
          bl.ld1 = d.ldp;
          bl.ld2 = d.ldp;
          bl.rows = r;
          bl.cols = r;
          bl.cbeg = (int32_t)scon.size();
          SchurContrib<T> sc{};
          sc.Xa = F + (size_t)nf * d.ldf;
          sc.Xb = sc.Xa;
          sc.lds = d.ldf;
          sc.ns = nf;
          sc.owner = d.p;
          scon.push_back(sc);
          bl.cend = (int32_t)scon.size();
          for (int i0 = 0; i0 < r; i0 += TB)
            for (int j0 = 0; j0 < r; j0 += TB) stiles.push_back({(int32_t)sblk.size(), i0, j0});
          sblk.push_back(bl);
          const double rr = r, ff = nf;
          fl += 2 * rr * rr * ff + 4 * ff * ff * rr;
        }
        const double rr = r, ff = nf;
        fl += ff * ff * ff / 3 + ff * ff * rr + ff * rr * rr;
      }
      {
        const double rr = r, np_ = d.np;
        fl += rr * rr * np_ - 2 * rr * rr * rr / 3 + nf * rr * rr;  // pivoted Cholesky, T_cf
      }
      h->st.mem_f += (int64_t)r * nf * 2 + (int64_t)nf * (nf + 1) / 2;
      hsz[d.p] = r;
    }
    rank_slot += nc;
    {
      Packer pk2;
      const size_t oi2 = pk2.add(it);
      const size_t oa = pk2.add(g12), ota = pk2.add(t12), ob = pk2.add(g3), otb = pk2.add(t3);
      void* d2 = upload<T>(h, pk2, s);
      if (!t12.empty()) {
        k_dgemm_sub<<<(unsigned)t12.size(), 256, 0, s>>>(at<const DGemmTask>(d2, oa), at<const DGemmTile>(d2, ota));
        CKLAUNCH();
        ++nl;
      }
      if (!t3.empty()) {
        k_dgemm_sub<<<(unsigned)t3.size(), 256, 0, s>>>(at<const DGemmTask>(d2, ob), at<const DGemmTile>(d2, otb));
        CKLAUNCH();
        ++nl;
      }
      // copies, then gathers: the warps of a task's CTAs take columns (about
      // eight each)
      int cols = 1;
      for (const InterpTask<T>& d : it) cols = std::max(cols, d.m + d.np);
      const dim3 grid((unsigned)std::min(32, (cols + 63) / 64), (unsigned)nc);
      k_interp_copy<T><<<grid, 256, 0, s>>>(at<const InterpTask<T>>(d2, oi2), d_nbrs, d_cur);
      CKLAUNCH();
      k_interp_store<T><<<grid, 256, 0, s>>>(at<const InterpTask<T>>(d2, oi2), d_nbrs, d_cur);
      CKLAUNCH();
      nl += 2;
    }
    h->st.factor_flops += fl;
    h->prof.launches += nl;
    h->prof.end(pid, s, fl, by, nl);
    // eliminate f: C_ff = U_f^T U_f, X_fc = U_f^{-T} C_fc, Y_f = U_f^{-T},
    // then A_cc -= X_fc^T X_fc
    set_identity<T>(h, ident, s);
    pivot_chol<T>(h, diag, d_finfo + c, s);
    trsm_batch<T>(h, tr, s);
    if (!stiles.empty()) {
      Packer pk3;
      const size_t ob = pk3.add(sblk), oc = pk3.add(scon), ot = pk3.add(stiles);
      void* d3 = upload<T>(h, pk3, s);
      const int spid = h->prof.begin(F_SCHUR, s);
      k_schur<T><<<(unsigned)stiles.size(), NT, 0, s>>>(at<const SchurTile>(d3, ot), at<const SchurBlock<T>>(d3, ob),
                                                       at<const SchurContrib<T>>(d3, oc));
      CKLAUNCH();
      h->prof.launches += 1;
      double bfl = 0, bby = 0;
      for (const auto& bl : sblk) {
        const double ns = scon[bl.cbeg].ns;
        bfl += 2.0 * bl.rows * bl.cols * ns;
        bby += ((double)(bl.rows + bl.cols) * ns + 2.0 * bl.rows * bl.cols) * sizeof(T);
      }
      h->prof.end(spid, s, bfl, bby, 1);
    }
  }
  return out;
}

// The subtractions x_v -= tmp[k] of an elimination phase's scatter, grouped
// by target slot v (appended to tslot / tptr / tidx): a stable counting sort,
// so each target's sources stay in op order (the fixed summation order).
// Few targets against many slots (the upper levels): a comparison sort on
// (slot, position) gives the same grouping and order without the O(n) passes.
static void group_by_target(spand_handle h, int64_t n, const std::vector<std::pair<int32_t, int64_t>>& tgt,
                            std::vector<int32_t>& tslot, std::vector<int64_t>& tptr, std::vector<int64_t>& tidx) {
  if ((double)tgt.size() * 32.0 < (double)n) {
    std::vector<std::pair<int32_t, int64_t>> key(tgt.size());
    for (size_t i = 0; i < tgt.size(); ++i) key[i] = {tgt[i].first, (int64_t)i};
    std::sort(key.begin(), key.end());
    tidx.reserve(tidx.size() + tgt.size());
    for (size_t i = 0; i < key.size();) {
      const int32_t v = key[i].first;
      tslot.push_back(v);
      for (; i < key.size() && key[i].first == v; ++i) tidx.push_back(tgt[(size_t)key[i].second].second);
      tptr.push_back((int64_t)tidx.size());
    }
    return;
  }
  std::vector<int64_t>& head = h->gb_head;
  head.assign((size_t)n + 1, 0);
  for (const auto& e : tgt) ++head[(size_t)e.first + 1];
  for (int64_t v = 0; v < n; ++v) head[v + 1] += head[v];
  std::vector<int64_t>& byslot = h->gb_byslot;
  byslot.resize(tgt.size());
  for (size_t i = 0; i < tgt.size(); ++i) byslot[head[tgt[i].first]++] = tgt[i].second;
  // head[v] is now the end of slot v's run
  tidx.reserve(tidx.size() + tgt.size());
  int64_t b = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t e = head[v];
    if (e == b) continue;
    tslot.push_back((int32_t)v);
    for (int64_t k = b; k < e; ++k) tidx.push_back(byslot[k]);
    tptr.push_back((int64_t)tidx.size());
    b = e;
  }
}

// One elimination op of the apply given by its factor blocks and slot lists:
// s (ns slots) is eliminated against n (m slots).
template <typename T>
struct ElimSpec {
  const T* XT;  // X^T, ns x m, leading dimension ld
  const T* Y;   // U_s^{-T} (ns x ns, ld ns), or nullptr for U_s = I
  int32_t ld;
  std::vector<int32_t> s_slots, n_slots;
};

// A phase group of the apply made of elimination ops only (its temporaries
// start at 0: the phases of one group are separated from every other
// group's by grid barriers, and nothing in tmp outlives a sweep through a
// group).  Uploaded to the persistent arena.
template <typename T>
static ApplyStep<T> make_elim_step(spand_handle h, const std::vector<ElimSpec<T>>& specs, cudaStream_t s) {
  std::vector<ElimOp<T>> eops;
  std::vector<int32_t> aslots, tslot;
  std::vector<int64_t> tptr(1, 0), tidx;
  std::vector<std::pair<int32_t, int64_t>> tgt;
  std::vector<ApplyItem> fy, fu, ba, bx;
  int64_t tmp_off = 0;
  for (const ElimSpec<T>& sp : specs) {
    ElimOp<T> o{};
    o.XT = sp.XT;
    o.Y = sp.Y;
    o.ld = sp.ld;
    o.ns = (int32_t)sp.s_slots.size();
    o.m = (int32_t)sp.n_slots.size();
    if (o.ns == 0) continue;
    o.slot = (int64_t)aslots.size();
    o.ty = tmp_off;
    o.tu = tmp_off + o.ns;
    o.ta = tmp_off + o.ns + o.m;
    const int32_t op = (int32_t)eops.size();
    aslots.insert(aslots.end(), sp.s_slots.begin(), sp.s_slots.end());
    aslots.insert(aslots.end(), sp.n_slots.begin(), sp.n_slots.end());
    for (int32_t i = 0; i < o.ns; ++i) {  // x_s = y_s
      tslot.push_back(sp.s_slots[i]);
      tidx.push_back(o.ty + i);
      tptr.push_back((int64_t)tidx.size());
    }
    for (int32_t k = 0; k < o.m; ++k) tgt.push_back({sp.n_slots[k], o.tu + k});
    for (int32_t r0 = 0; r0 < o.ns; r0 += RB) {
      fy.push_back({op, r0});
      ba.push_back({op, r0});
    }
    for (int32_t c0 = 0; c0 < o.m; c0 += AP_COLS) fu.push_back({op, c0});
    for (int32_t c0 = 0; c0 < o.ns; c0 += AP_COLS) bx.push_back({op, c0});
    tmp_off += 2 * (int64_t)o.ns + o.m;
    eops.push_back(o);
  }
  ApplyStep<T> ap;
  if (eops.empty()) return ap;
  h->tmp_len = std::max(h->tmp_len, tmp_off);
  const int64_t nassign = (int64_t)tslot.size();
  group_by_target(h, h->n, tgt, tslot, tptr, tidx);
  Packer pk;
  const size_t oe = pk.add(eops), osl = pk.add(aslots), ots = pk.add(tslot), otp = pk.add(tptr), oti = pk.add(tidx);
  const size_t ofy = pk.add(fy), ofu = pk.add(fu), oba = pk.add(ba), obx = pk.add(bx);
  void* d = h->persist.alloc(pk.size);
  void* src = h->stage.take(pk.size);
  pk.write(src);
  CK(cudaMemcpyAsync(d, src, pk.size, cudaMemcpyHostToDevice, s));
  ap.n_elim = (int)eops.size();
  ap.elim = at<const ElimOp<T>>(d, oe);
  ap.slots = at<const int32_t>(d, osl);
  ap.ntgt = (int64_t)tslot.size();
  ap.nassign = nassign;
  ap.tslot = at<const int32_t>(d, ots);
  ap.tptr = at<const int64_t>(d, otp);
  ap.tidx = at<const int64_t>(d, oti);
  ap.n_fy = (int)fy.size();
  ap.n_fu = (int)fu.size();
  ap.n_ba = (int)ba.size();
  ap.n_bx = (int)bx.size();
  ap.fy = at<const ApplyItem>(d, ofy);
  ap.fu = at<const ApplyItem>(d, ofu);
  ap.ba = at<const ApplyItem>(d, oba);
  ap.bx = at<const ApplyItem>(d, obx);
  return ap;
}

// The apply program: the phases of every step in execution order (forward
// sweep leaves -> root, then the backward sweep root -> leaves), uploaded once
// per factorization, and the cooperative grid that runs it.
template <typename TF>
static void build_apply_program(spand_handle h, const std::vector<ApplyStep<TF>>& steps, cudaStream_t s) {
  std::vector<ApplyPhase<TF>> ph;
  auto items = [&](int32_t kind, const ApplyStep<TF>& a, const ApplyItem* it, int n) {
    if (n <= 0) return;
    ApplyPhase<TF> p = {};
    p.kind = kind;
    p.n = n;
    p.elim = a.elim;
    p.sq = a.sq;
    p.items = it;
    p.slots = a.slots;
    ph.push_back(p);
  };
  for (const ApplyStep<TF>& a : steps) {
    if (a.n_elim) {
      items(PH_FY, a, a.fy, a.n_fy);
      items(PH_FU, a, a.fu, a.n_fu);
      if (a.ntgt > 0) {
        ApplyPhase<TF> p = {};
        p.kind = PH_SCATTER;
        p.n = (int32_t)a.ntgt;
        p.tslot = a.tslot;
        p.tptr = a.tptr;
        p.tidx = a.tidx;
        p.nassign = a.nassign;
        ph.push_back(p);
      }
    }
    if (a.n_sq) {
      items(PH_SY, a, a.sy, a.n_sy);
      items(PH_SC, a, a.sc, a.n_sc);
    }
  }
  for (auto it = steps.rbegin(); it != steps.rend(); ++it) {
    const ApplyStep<TF>& a = *it;
    if (a.n_sq) {
      items(PH_SZ, a, a.sz, a.n_sz);
      items(PH_SX, a, a.sx, a.n_sx);
    }
    if (a.n_elim) {
      items(PH_BA, a, a.ba, a.n_ba);
      items(PH_BX, a, a.bx, a.n_bx);
    }
  }
  h->n_aprog = (int)ph.size();
  h->aprog = nullptr;
  if (!ph.empty()) {
    void* d = h->persist.alloc(ph.size() * sizeof(ApplyPhase<TF>));
    void* src = h->stage.take(ph.size() * sizeof(ApplyPhase<TF>));
    std::memcpy(src, ph.data(), ph.size() * sizeof(ApplyPhase<TF>));
    CK(cudaMemcpyAsync(d, src, ph.size() * sizeof(ApplyPhase<TF>), cudaMemcpyHostToDevice, s));
    h->aprog = d;
  }
  h->d_bar.ensure(2 * sizeof(unsigned));
  CK(cudaMemsetAsync(h->d_bar.p, 0, 2 * sizeof(unsigned), s));
  const void* fn = (const void*)k_apply<TF>;
  h->apply_smem = (size_t)SCH * sizeof(TF) + ph.size() * sizeof(ApplyPhase<TF>);
  ensure_smem(fn, h->apply_smem);
  int dev = 0, nsm = 0, coop = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) throw Fail{SPAND_ERR_CUDA, "device does not support cooperative launches (needed by the apply)"};
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_apply<TF>, AT, h->apply_smem));
  if (per_sm < 1) throw Fail{SPAND_ERR_CUDA, "apply kernel cannot be resident"};
  h->apply_per_sm_max = std::min(per_sm, kApplyCtasPerSm);
  h->apply_grid = nsm * (h->apply_ctas > 0 ? std::min(h->apply_ctas, h->apply_per_sm_max) : h->apply_per_sm_max);
}

template <typename T>
static int factorize_impl(spand_handle h, cudaStream_t s) {
  const Tree& tr = h->tree;
  const int L = tr.L;
  const double eps = h->opts.eps;
  const int skip = h->opts.skip;
  h->persist.reset();
  h->descs.reset();
  std::vector<ApplyStep<T>> apply;
  h->sizes_before.assign(L, {});
  h->sizes_after.assign(L, {});
  for (double& v : h->phase_ms) v = 0;
  spand_stats& stt = h->st;
  stt.size_top = 0;
  stt.mem_f = 0;
  stt.factor_flops = 0;
  stt.fail_step = 0;
  stt.fail_cluster = -1;
  StepTimer tm(L);
  h->stage.reset();  // the previous factorization ended with a stream synchronisation
  // non-positive pivot flags per step: [2t] elimination pivots, [2t+1]
  // scaling pivots ([0]: a bounded device wait gave up);
  // read at the next host synchronisation (the rank readback of a
  // sparsifying step, or the end of the factorization)
  // (then, for the interpolative variants, one flag per step and colour for
  // the f blocks C_ff)
  int maxcol = 1;
  for (const StepStruct& sx : tr.steps) maxcol = std::max(maxcol, sx.ncolours());
  const size_t ninfo = 2 * (size_t)(L + 1) + (size_t)(L + 1) * maxcol;
  int* d_info = (int*)h->descs.alloc(ninfo * sizeof(int));
  CK(cudaMemsetAsync(d_info, 0, ninfo * sizeof(int), s));
  std::vector<std::vector<int>> elim_cls(L + 1), scale_cls(L + 1);  // cluster of each pivot-batch entry
  std::vector<std::vector<std::vector<int>>> f_cls(L + 1);           // per step and colour: the f blocks' interfaces
  auto check_pivots = [&](int upto) {  // after a stream synchronisation
    std::vector<int> info(ninfo, 0);
    CK(cudaMemcpy(info.data(), d_info, info.size() * sizeof(int), cudaMemcpyDeviceToHost));
    if (info[0])
      throw Fail{SPAND_ERR_TIMEOUT, "Schur update: a bounded tensor-core wait (MMA completion or operand "
                                    "copy) timed out"};
    for (int u = 1; u <= upto; ++u) {
      if (info[2 * u] || info[2 * u + 1]) {
        stt.fail_step = u;
        stt.fail_cluster = info[2 * u] ? elim_cls[u][info[2 * u] - 1] : scale_cls[u][info[2 * u + 1] - 1];
        throw Fail{SPAND_ERR_NOT_SPD, std::string(info[2 * u] ? "pivot" : "interface") +
                                          " block not positive definite at step " + std::to_string(u)};
      }
      for (int c = 0; c < (int)f_cls[u].size() && c < maxcol; ++c) {
        const int v = info[2 * (size_t)(L + 1) + (size_t)u * maxcol + c];
        if (v) {
          stt.fail_step = u;
          stt.fail_cluster = f_cls[u][c][v - 1];
          throw Fail{SPAND_ERR_NOT_SPD, "interpolative sparsification: block C_ff not positive definite at step " +
                                            std::to_string(u)};
        }
      }
    }
  };

  const int nc0 = (int)tr.cluster_ptr.size() - 1;
  std::vector<int32_t> sz(nc0);
  std::vector<std::vector<int32_t>> slots(nc0);
  for (int i = 0; i < nc0; ++i) {
    sz[i] = tr.cluster_ptr[i + 1] - tr.cluster_ptr[i];
    slots[i].resize(sz[i]);
    std::iota(slots[i].begin(), slots[i].end(), tr.cluster_ptr[i]);
  }
  CK(cudaEventRecord(tm.at(0, 0), s));
  Layout<T> lay = make_layout<T>(h, 1, sz, s);
  {  // assemble A into the step-1 rows
    Packer pk;
    size_t orow = pk.add(lay.row);
    void* d = upload<T>(h, pk, s);
    const int64_t nnz = h->nnz;
    if (nnz > 0) {
      const int g = (int)std::min<int64_t>((nnz + 255) / 256, 4096);
      k_assemble<T><<<g, 256, 0, s>>>((const double*)h->d_vals.p, (const int32_t*)h->d_asm_row.p,
                                      (const int64_t*)h->d_asm_off.p, at<T* const>(d, orow), nnz);
      CKLAUNCH();
      h->prof.launches += 1;
    }
  }
  CK(cudaEventRecord(tm.at(0, 1), s));

  int32_t* d_cur = nullptr;
  std::function<void()> pending;  // the previous step's deferred apply-program build
  auto run_pending = [&]() {
    if (pending) {
      auto f = std::move(pending);
      pending = nullptr;
      f();
    }
  };
  std::vector<std::vector<int32_t>> slots_of_step;
  for (int t = 1; t <= L; ++t) {
    const StepStruct& st = tr.steps[t - 1];
    const int n = st.n;
    h->sizes_before[t - 1] = sz;
    if (t == L)
      for (int i = 0; i < n; ++i)
        if (st.elim[i]) stt.size_top += sz[i];
    CK(cudaEventRecord(tm.at(t, 0), s));
    // ------------------------------------------------ eliminate (Sec. 2.4)
    std::vector<int> seps, rems;
    for (int i = 0; i < n; ++i) (st.elim[i] ? seps : rems).push_back(i);
    std::vector<T*> ysep(n, nullptr);
    {
      std::vector<RowDesc<T>> diag, ident;
      std::vector<int> diag_cl;
      std::vector<double> diag_fl, tr_fl;
      std::vector<TrsmTask<T>> tr_tasks;
      for (int sidx : seps) {
        if (sz[sidx] <= 0) continue;
        const double ns = sz[sidx], m = lay.W[sidx] - sz[sidx];
        // step 1: the pivot is a piece of A, with the envelope found at analysis
        const bool env = t == 1 && !h->env_bw.empty();
        const int bw = env ? h->env_bw[sidx] : 0, bw2 = env ? h->env_bw32[sidx] : 0;
        const int band = env ? h->env_band[sidx] : 0;
        const double cfl = env ? h->env_flops[sidx] : ns * ns * ns / 3;
        const double nnzU = env ? h->env_nnz[sidx] : ns * (ns + 1) / 2;
        T* dv = alloc_dinv<T>(h, sz[sidx]);
        diag.push_back({lay.row[sidx], sz[sidx], lay.ld[sidx], dv, bw, bw2, band, 0});
        diag_cl.push_back(sidx);
        diag_fl.push_back(cfl);
        add_panels(tr_tasks, lay.row[sidx], (const T*)dv, sz[sidx], lay.ld[sidx], sz[sidx], lay.W[sidx], bw, &tr_fl,
                   nnzU);
        T* Y = (T*)h->persist.alloc((size_t)sz[sidx] * sz[sidx] * sizeof(T));
        ysep[sidx] = Y;
        ident.push_back({Y, sz[sidx], sz[sidx], nullptr, 0, 0});
        add_inverse(tr_tasks, (const T*)lay.row[sidx], (const T*)dv, sz[sidx], lay.ld[sidx], Y, bw, &tr_fl);
        stt.factor_flops += cfl + 2 * nnzU * m + ns * m * m;
      }
      set_identity<T>(h, ident, s);
      pivot_chol<T>(h, diag, d_info + 2 * t, s, &diag_fl);
      elim_cls[t] = diag_cl;
      trsm_batch<T>(h, tr_tasks, s, &tr_fl);
      // pull-form Schur update of every pair of neighbours: target blocks in
      // the order of their first contribution (separators in order, then
      // their neighbour pairs), each with its contributions in separator
      // order; clusters reduced to nothing are left out
      if (h->splan.size() < (size_t)L + 1) h->splan.resize((size_t)L + 1);
      auto& plan = h->splan[t];
      if (!plan.built) {
        std::unordered_map<int64_t, int32_t> bid;
        std::vector<std::vector<int32_t>> cl;  // per block: contribution triples (sep, ea, eb)
        for (int sidx : seps) {
          const int32_t nb0 = lay.nptr[sidx], nb1 = lay.nptr[sidx + 1];
          for (int32_t ea = nb0; ea < nb1; ++ea)
            for (int32_t eb = ea; eb < nb1; ++eb) {
              const int32_t a = lay.nidx[ea], b = lay.nidx[eb];
              const int64_t key = (int64_t)a * n + b;
              auto it = bid.find(key);
              int32_t id;
              if (it == bid.end()) {
                id = (int32_t)plan.a.size();
                bid.emplace(key, id);
                const int32_t eab = a == b ? -1 : lay.edge_of(a, b), eba = a == b ? -1 : lay.edge_of(b, a);
                if (a != b && (eab < 0 || eba < 0)) throw Fail{SPAND_ERR_STATE, "fill block missing from the layout"};
                plan.a.push_back(a);
                plan.b.push_back(b);
                plan.eab.push_back(eab);
                plan.eba.push_back(eba);
                cl.emplace_back();
              } else {
                id = it->second;
              }
              cl[id].insert(cl[id].end(), {sidx, ea, eb});
            }
        }
        plan.cptr.assign(1, 0);
        for (const auto& v : cl) {
          for (size_t k = 0; k < v.size(); k += 3) {
            plan.csep.push_back(v[k]);
            plan.cea.push_back(v[k + 1]);
            plan.ceb.push_back(v[k + 2]);
          }
          plan.cptr.push_back((int32_t)plan.csep.size());
        }
        plan.built = true;
      }
      std::vector<SchurBlock<T>> blocks;
      std::vector<SchurContrib<T>> flat;
      blocks.reserve(plan.a.size());
      flat.reserve(plan.csep.size());
      for (size_t id = 0; id < plan.a.size(); ++id) {
        const int32_t a = plan.a[id], b = plan.b[id];
        if (sz[a] <= 0 || sz[b] <= 0) continue;
        const int32_t cb = (int32_t)flat.size();
        for (int32_t k = plan.cptr[id]; k < plan.cptr[id + 1]; ++k) {
          const int32_t sidx = plan.csep[k];
          if (sz[sidx] <= 0) continue;
          SchurContrib<T> c;
          c.Xa = lay.row[sidx] + (size_t)lay.noff[plan.cea[k]] * lay.ld[sidx];
          c.Xb = lay.row[sidx] + (size_t)lay.noff[plan.ceb[k]] * lay.ld[sidx];
          c.lds = lay.ld[sidx];
          c.ns = sz[sidx];
          c.owner = sidx;
          flat.push_back(c);
        }
        if ((int32_t)flat.size() == cb) continue;
        SchurBlock<T> bl;
        bl.C1 = lay.row[a] + (size_t)(a == b ? 0 : lay.noff[plan.eab[id]]) * lay.ld[a];
        bl.C2 = (a == b) ? nullptr : lay.row[b] + (size_t)lay.noff[plan.eba[id]] * lay.ld[b];
        bl.ld1 = lay.ld[a];
        bl.ld2 = lay.ld[b];
        bl.rows = sz[a];
        bl.cols = sz[b];
        bl.cbeg = cb;
        bl.cend = (int32_t)flat.size();
        blocks.push_back(bl);
      }
      if (!blocks.empty()) {
        std::vector<SchurTile> tiles;
        // tensor cores for the TF32 / BF16 forms: 128 x 64 tiles; FP32 and
        // FP64 on the SIMT pipes: 64 x 64 tiles
        bool tc = sizeof(T) == 4 && (h->opts.precision == SPAND_TF32 || h->opts.precision == SPAND_BF16);
        for (size_t k = 0; tc && k < flat.size(); ++k) {  // the kernel loads 16-byte vectors of X
          const SchurContrib<T>& c = flat[k];
          if (c.lds % 4 != 0 || ((uintptr_t)c.Xa | (uintptr_t)c.Xb) % 16 != 0) tc = false;
        }
        // TF32: operands through the copy engine (one tensor map pair per
        // separator row); BF16 converts in registers (k_schur_tc)
        std::vector<CUtensorMap> tmaps;
        std::vector<int32_t> tmap_of(n, -1);
        bool tma = tc && h->opts.precision == SPAND_TF32 && tmap_encoder() != nullptr;
        for (int sidx : seps) {
          if (!tma) break;
          if (sz[sidx] <= 0 || lay.nptr[sidx + 1] == lay.nptr[sidx]) continue;
          tmap_of[sidx] = (int32_t)tmaps.size();
          tmaps.resize(tmaps.size() + 2);
          if (!encode_row_map(&tmaps[tmaps.size() - 2], (const float*)lay.row[sidx], sz[sidx], lay.W[sidx],
                              lay.ld[sidx], TC_M) ||
              !encode_row_map(&tmaps[tmaps.size() - 1], (const float*)lay.row[sidx], sz[sidx], lay.W[sidx],
                              lay.ld[sidx], TC_N))
            tma = false;
        }
        const int ti = tc ? TC_M : TB, tj = tc ? TC_N : TB;
        for (size_t b = 0; b < blocks.size(); ++b) {
          for (int i0 = 0; i0 < blocks[b].rows; i0 += ti)
            for (int j0 = 0; j0 < blocks[b].cols; j0 += tj) tiles.push_back({(int32_t)b, i0, j0});
        }
        const CUtensorMap* dmaps = nullptr;
        if (tma) {
          Packer pkm;
          const size_t om = pkm.add(tmaps);
          dmaps = at<const CUtensorMap>(upload<T>(h, pkm, s), om);
        }
        std::vector<SchurContribTma> flat_tma;
        if (tma) {
          flat_tma.reserve(flat.size());
          for (const SchurContrib<T>& c : flat) {
            // the separator row is the one whose columns Xa, Xb point into
            const int sidx = c.owner;
            SchurContribTma m{};
            m.map_a = dmaps + tmap_of[sidx];
            m.map_b = dmaps + tmap_of[sidx] + 1;
            m.col_a = (int32_t)((c.Xa - lay.row[sidx]) / lay.ld[sidx]);
            m.col_b = (int32_t)((c.Xb - lay.row[sidx]) / lay.ld[sidx]);
            m.ns = c.ns;
            flat_tma.push_back(m);
          }
        }
        Packer pk;
        size_t ob = pk.add(blocks), oc = tma ? pk.add(flat_tma) : pk.add(flat), ot = pk.add(tiles);
        void* d = upload<T>(h, pk, s);
        double fl = 0, by = 0;
        for (auto& bl : blocks) {
          double ksum = 0;
          for (int32_t c = bl.cbeg; c < bl.cend; ++c) ksum += flat[c].ns;
          fl += 2.0 * bl.rows * bl.cols * ksum;
          by += ((double)(bl.rows + bl.cols) * ksum + (bl.C2 ? 3.0 : 2.0) * bl.rows * bl.cols) * sizeof(T);
        }
        const int pid = h->prof.begin(F_SCHUR, s);
        if constexpr (sizeof(T) == 4) {
          if (tma) {
            const void* fn = (const void*)k_schur_tma;
            ensure_smem(fn, TM_SMEM);
            const SchurTile* a0 = at<const SchurTile>(d, ot);
            const SchurBlock<float>* a1 = at<const SchurBlock<float>>(d, ob);
            const SchurContribTma* a2 = at<const SchurContribTma>(d, oc);
            int* a3 = d_info;  // [0]: a bounded wait gave up
            void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3};
            CK(cudaLaunchKernel(fn, dim3((unsigned)tiles.size()), dim3(TC_NT), args, TM_SMEM, s));
          } else if (tc) {
            const void* fn = h->opts.precision == SPAND_BF16 ? (const void*)k_schur_tc<true> : (const void*)k_schur_tc<false>;
            const size_t tsm = TC_SMEM;
            ensure_smem(fn, tsm);
            const SchurTile* a0 = at<const SchurTile>(d, ot);
            const SchurBlock<float>* a1 = at<const SchurBlock<float>>(d, ob);
            const SchurContrib<float>* a2 = at<const SchurContrib<float>>(d, oc);
            int* a3 = d_info;  // [0]: a bounded tensor-core wait gave up
            void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3};
            CK(cudaLaunchKernel(fn, dim3((unsigned)tiles.size()), dim3(TC_NT), args, tsm, s));
          }
        }
        if (!tc)
          k_schur<T><<<(unsigned)tiles.size(), NT, 0, s>>>(at<const SchurTile>(d, ot), at<const SchurBlock<T>>(d, ob),
                                                          at<const SchurContrib<T>>(d, oc));
        CKLAUNCH();
        h->prof.launches += 1;
        h->prof.end(pid, s, fl, by, 1);
      }
    }
    CK(cudaEventRecord(tm.at(t, 1), s));
    // ------------------------------------------------ apply ops of the elimination
    ApplyStep<T> ap;
    std::vector<int32_t> aslots = h->pool32.take();
    std::vector<ElimOp<T>> eops;
    std::vector<std::pair<int32_t, int64_t>> tgt = h->poolpair.take();  // (target slot, tmp index) of the subtractions
    std::vector<int32_t> tslot = h->pool32.take();
    std::vector<int64_t> tptr = h->pool64.take(), tidx = h->pool64.take();
    tptr.push_back(0);
    std::vector<ApplyItem> it_fy = h->poolitem.take(), it_fu = h->poolitem.take(), it_ba = h->poolitem.take(),
                           it_bx = h->poolitem.take();
    int64_t tmp_off = 0;
    size_t sm_ns = 0, sm_m = 0;
    int64_t nassign = 0;
    bool elim_ops_built = false;
    // built after the sparsification launches (its host time then overlaps them)
    auto build_elim_ops = [&]() {
      for (int sidx : seps) {
        if (sz[sidx] <= 0) continue;
        ElimOp<T> o{};
        o.XT = lay.row[sidx] + (size_t)lay.ld[sidx] * sz[sidx];
        o.ld = lay.ld[sidx];
        o.Y = ysep[sidx];
        o.ns = sz[sidx];
        o.m = lay.W[sidx] - sz[sidx];
        o.slot = (int64_t)aslots.size();
        o.ty = tmp_off;
        o.tu = tmp_off + o.ns;
        o.ta = tmp_off + o.ns + o.m;
        const int32_t op = (int32_t)eops.size();
        aslots.insert(aslots.end(), slots[sidx].begin(), slots[sidx].end());
        for (int32_t i = 0; i < o.ns; ++i) {  // x_s = y_s
          tslot.push_back(slots[sidx][i]);
          tidx.push_back(o.ty + i);
          tptr.push_back((int64_t)tidx.size());
        }
        int64_t j = 0;
        for (int32_t e = lay.nptr[sidx]; e < lay.nptr[sidx + 1]; ++e) {
          const int32_t q = lay.nidx[e];
          for (int32_t k = 0; k < sz[q]; ++k, ++j) {
            aslots.push_back(slots[q][k]);
            tgt.push_back({slots[q][k], o.tu + j});
          }
        }
        for (int32_t r0 = 0; r0 < o.ns; r0 += RB) {
          it_fy.push_back({op, r0});
          it_ba.push_back({op, r0});
        }
        for (int32_t c0 = 0; c0 < o.m; c0 += AP_COLS) it_fu.push_back({op, c0});
        for (int32_t c0 = 0; c0 < o.ns; c0 += AP_COLS) it_bx.push_back({op, c0});
        tmp_off += 2 * (int64_t)o.ns + o.m;
        eops.push_back(o);
        stt.mem_f += (int64_t)o.ns * (o.ns + 1) / 2 + (int64_t)o.ns * o.m;
        sm_ns = std::max(sm_ns, (size_t)o.ns * sizeof(double));
        sm_m = std::max(sm_m, (size_t)o.m * sizeof(double));
      }
      h->tmp_len = std::max(h->tmp_len, tmp_off);
      nassign = (int64_t)tslot.size();
      group_by_target(h, h->n, tgt, tslot, tptr, tidx);
      h->poolpair.give(std::move(tgt));
      elim_ops_built = true;
    };

    // ------------------------------------------------ scale + sparsify
    std::vector<int32_t> sz_after = sz;
    for (int sidx : seps) sz_after[sidx] = 0;
    std::vector<SqOp<T>> sqops;
    std::vector<int> sq_cluster;
    std::vector<int> cp_index;  // per cluster: index in cp_cluster, -1 if not sparsified
    size_t sm_np = 0, sm_r = 0;
    const bool sparsify = (skip < t) && (t < L);
    int cpqr_pid = -1;
    std::vector<int> ell_fin;              // randomized compression: final sketch width per task
    std::vector<InterpOut<T>> interp_out;  // interpolative variants: per task
    std::vector<std::vector<int32_t>> kept_slots(n);  // and the slots each interface keeps
    std::vector<char> has_kept(n, 0);
    std::vector<ApplyStep<T>> interp_steps;  // their apply groups: T_p ops, then the eliminations of f
    std::vector<int> cp_cluster;           // sparsified clusters (task order)
    std::vector<T*> cp_qc;                 // their Q_pc scratch
    if (sparsify) {
      std::vector<RowDesc<T>> diag, ident;
      std::vector<int> diag_cl;
      std::vector<TrsmTask<T>> up;
      std::vector<CopyTask<T>> m_up, m_lo;  // per pair p < q: p -> q (the product's operands), q -> p
      std::vector<RowDesc<T>> idr;
      for (int p : rems) {
        if (sz[p] <= 0 || h->opts.variant == SPAND_IN) continue;  // In: no block scaling
        T* dv = alloc_dinv<T>(h, sz[p]);
        diag.push_back({lay.row[p], sz[p], lay.ld[p], dv});
        diag_cl.push_back(p);
        const int fu = lay.first_upper(p);
        add_panels(up, lay.row[p], (const T*)dv, sz[p], lay.ld[p], fu, lay.W[p]);
        for (int32_t e = lay.nptr[p]; e < lay.nptr[p + 1]; ++e) {
          const int32_t q = lay.nidx[e];
          if (q <= p || sz[q] <= 0) continue;
          const int32_t oqp = lay.off_of(q, p);
          CopyTask<T> c;
          c.src = lay.row[p] + (size_t)lay.noff[e] * lay.ld[p];
          c.dst = lay.row[q] + (size_t)oqp * lay.ld[q];
          c.lds = lay.ld[p];
          c.ldd = lay.ld[q];
          c.rows = sz[q];
          c.cols = sz[p];
          c.trans = 1;
          c.pad = 0;
          m_up.push_back(c);
          CopyTask<T> b = c;
          b.src = c.dst;
          b.dst = const_cast<T*>(c.src);
          b.lds = lay.ld[q];
          b.ldd = lay.ld[p];
          b.rows = sz[p];
          b.cols = sz[q];
          m_lo.push_back(b);
        }
        T* Y = (T*)h->persist.alloc((size_t)sz[p] * sz[p] * sizeof(T));
        ident.push_back({Y, sz[p], sz[p], nullptr});
        add_inverse(up, (const T*)lay.row[p], (const T*)dv, sz[p], lay.ld[p], Y);
        idr.push_back({lay.row[p], sz[p], lay.ld[p], nullptr});
        SqOp<T> so{};
        so.Y = Y;
        so.Q = nullptr;
        so.np = sz[p];
        so.r = sz[p];
        sqops.push_back(so);
        sq_cluster.push_back(p);
        const double np_ = sz[p], m = lay.W[p] - sz[p];
        stt.factor_flops += np_ * np_ * np_ / 3 + np_ * np_ * m;
        stt.mem_f += (int64_t)sz[p] * (sz[p] + 1) / 2;
        sm_np = std::max(sm_np, (size_t)sz[p] * sizeof(double));
      }
      // second side of every pair p < q from the first side's block and Y_q:
      // O = Y_q (U_p^{-T} A_pq)^T into q's row (the scaled A_qp)
      std::vector<ScaleTask<T>> sct;
      std::vector<SchurTile> sctl;
      {
        std::vector<const T*> yof(n, nullptr);
        for (size_t i = 0; i < sq_cluster.size(); ++i) yof[sq_cluster[i]] = sqops[i].Y;
        for (const CopyTask<T>& c : m_up) {  // one per pair p < q: src = p's block, dst = q's block
          ScaleTask<T> k;
          k.B = c.src;
          k.O = c.dst;
          k.ldb = c.lds;
          k.ldo = c.ldd;
          k.np = c.cols;
          k.nq = c.rows;
          k.Y = nullptr;
          sct.push_back(k);
        }
        size_t i = 0;
        for (int p : rems) {
          if (sz[p] <= 0 || h->opts.variant == SPAND_IN) continue;
          for (int32_t e = lay.nptr[p]; e < lay.nptr[p + 1]; ++e) {
            const int32_t q = lay.nidx[e];
            if (q <= p || sz[q] <= 0) continue;
            sct[i++].Y = yof[q];
          }
        }
        for (size_t k = 0; k < sct.size(); ++k)
          for (int i0 = 0; i0 < sct[k].nq; i0 += TB)
            for (int j0 = 0; j0 < sct[k].np; j0 += TB) sctl.push_back({(int32_t)k, i0, j0});
      }
      set_identity<T>(h, ident, s);
      pivot_chol<T>(h, diag, d_info + 2 * t + 1, s);
      scale_cls[t] = diag_cl;
      trsm_batch<T>(h, up, s);   // upper blocks U_p^{-T} A_pq and the inverses Y_p
      if (!sctl.empty()) {
        Packer pks;
        const size_t okt = pks.add(sct), okl = pks.add(sctl);
        void* dks = upload<T>(h, pks, s);
        double fl = 0;
        for (const ScaleTask<T>& k : sct) fl += (double)k.nq * k.nq * k.np;
        const int pid = h->prof.begin(F_TRSM, s);
        k_scale_gemm<T><<<(unsigned)sctl.size(), NT, 0, s>>>(at<const SchurTile>(dks, okl),
                                                             at<const ScaleTask<T>>(dks, okt));
        CKLAUNCH();
        h->prof.launches += 1;
        h->prof.end(pid, s, fl, 0.0, 1);
      }
      copy_batch<T>(h, m_lo, s);
      set_identity<T>(h, idr, s);
      CK(cudaEventRecord(tm.at(t, 2), s));
      // ---- sparsify, colour by colour (Sec. 2.6.1)
      d_cur = (int32_t*)h->descs.alloc((size_t)n * sizeof(int32_t));
      {
        int32_t* src = (int32_t*)h->stage.take((size_t)n * sizeof(int32_t));
        std::copy(sz.begin(), sz.end(), src);
        CK(cudaMemcpyAsync(d_cur, src, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      }
      // simultaneous order: all interfaces in one launch, compressed from the
      // same matrix; ranks go to d_rank so that the sizes the kernels read
      // (d_cur) stay those of the scaled matrix until the launch is over
      const bool sim = h->opts.sparsify_order == SPAND_SIMULTANEOUS;
      const bool interp = h->opts.variant != SPAND_ORTHS;
      int32_t* d_rank = nullptr;
      if (sim) {
        d_rank = (int32_t*)h->descs.alloc((size_t)n * sizeof(int32_t));
        CK(cudaMemcpyAsync(d_rank, d_cur, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      }
      auto colour_of = [&](int p) { return sim ? 0 : (int)st.colour[p]; };
      std::vector<CpqrTask<T>> tasks;
      std::vector<CpqrNbr<T>> nbrs;
      std::vector<int> tclass;  // cluster size of each task
      std::vector<int> tres;    // 1: the task's chunk lives in shared memory
      std::vector<int> treg;    // lane-group size of the register-resident kernel (0: chunked kernel)
      const int ncol = st.ncolours();
      size_t wbytes = 0;
      struct WOff { size_t nrm, v, tau, qc, gw; };
      std::vector<WOff> woff;
      const size_t CB = kCpqrChunkBudget;
      const int max_cluster = cpqr_max_cluster<T>();
      for (int p : rems) {
        if (sz[p] <= 0) continue;
        if (lay.nptr[p + 1] == lay.nptr[p]) continue;  // no neighbours: nothing to compress against
        CpqrTask<T> tk{};
        tk.p = p;
        tk.np = sz[p];
        tk.ldp = lay.ld[p];
        tk.Rp = lay.row[p];
        tk.nbeg = (int32_t)nbrs.size();
        int mm = 0;
        for (int32_t e = lay.nptr[p]; e < lay.nptr[p + 1]; ++e) {
          const int32_t q = lay.nidx[e];
          CpqrNbr<T> nb;
          nb.Rq = lay.row[q];
          nb.q = q;
          nb.off_pq = lay.noff[e];
          nb.off_qp = lay.off_of(q, p);
          if (nb.off_qp < 0) throw Fail{SPAND_ERR_STATE, "asymmetric block pattern"};
          nb.ldq = lay.ld[q];
          nbrs.push_back(nb);
          mm += sz[q];
        }
        tk.nend = (int32_t)nbrs.size();
        tk.m_max = mm;
        tk.rank_out = d_rank;
        tk.nowb = sim ? 1 : 0;
        // smallest cluster whose per-CTA chunk fits in shared memory, and at
        // most ~2 columns per thread
        const size_t Lp = (size_t)cq_ld<T>(sz[p]);
        const int nnb_p = tk.nend - tk.nbeg;
        // shared memory of a CTA with its chunk resident, for cluster size c
        auto res_smem = [&](int c) {
          const int cp = (mm + c - 1) / c;
          return cq_fixed_smem<T>(nnb_p, sz[p], cp, c) + Lp * cp * sizeof(T);
        };
        int C = max_cluster;
        for (int c = 1; c <= max_cluster; c *= 2)
          if (res_smem(c) <= CB) { C = c; break; }
        while (C < max_cluster && (mm + C - 1) / C > 2 * CQ_MAXNT) C *= 2;
        if (!interp && (mm + C - 1) / C > CQ_CPT * CQ_MAXNT)
          throw Fail{SPAND_ERR_INVALID_ARG, "interface coupling too wide for the sparsification kernel (" +
                                                std::to_string(mm) + " columns)"};
        const bool resident = res_smem(C) <= CB;
        WOff w;
        w.nrm = 0;
        w.v = wbytes; wbytes += align256((size_t)sz[p] * sz[p] * sizeof(T));
        w.tau = wbytes; wbytes += align256((size_t)sz[p] * sizeof(T));
        w.qc = wbytes; wbytes += align256((size_t)sz[p] * sz[p] * sizeof(T));
        w.gw = wbytes;
        if (!resident && !interp) wbytes += align256((size_t)C * Lp * ((mm + C - 1) / C) * sizeof(T));
        woff.push_back(w);
        tasks.push_back(tk);
        tclass.push_back(C);
        tres.push_back(resident ? 1 : 0);
        treg.push_back(0);
        cp_cluster.push_back(p);
      }
      // Colours whose interfaces all fit in one wave of register-resident
      // clusters run on that kernel (FP32 factors only): its reflector steps
      // are cheaper, but its CTAs fill whole SMs, so a colour that would need
      // a second wave keeps the chunked kernel.
      if (sizeof(T) == 4 && !tasks.empty() && !interp) {
        std::vector<int> rg(tasks.size(), 0), rc(tasks.size(), 0);
        for (size_t i = 0; i < tasks.size(); ++i) {
          int G = 1;
          while (G * kCqrRows < tasks[i].np && G < 8) G *= 2;
          const int C = (tasks[i].m_max + kCqrThreads / G - 1) / (kCqrThreads / G);
          if (G * kCqrRows >= tasks[i].np && C >= 1 && C <= kCqrMaxCluster) rg[i] = G, rc[i] = C;
        }
        const int nc_ = sim ? 1 : std::max(ncol, 1);
        std::vector<int> need(nc_, 0), cap(nc_, INT_MAX);
        std::vector<char> ok(nc_, 1);
        int capc[4][kCqrMaxCluster + 1];  // SMs of one wave, per (G, C), looked up once
        for (auto& row : capc)
          for (int& v : row) v = -1;
        for (size_t i = 0; i < tasks.size(); ++i) {
          const int c = colour_of(tasks[i].p);
          if (!ok[c]) continue;
          if (!rg[i]) { ok[c] = 0; continue; }
          need[c] += rc[i];
          int& cc = capc[rg[i] == 1 ? 0 : rg[i] == 2 ? 1 : rg[i] == 4 ? 2 : 3][rc[i]];
          if (cc < 0) cc = cpqr_reg_capacity<T>(rg[i], rc[i]) * rc[i];
          cap[c] = std::min(cap[c], cc);
        }
        for (size_t i = 0; i < tasks.size(); ++i) {
          const int c = colour_of(tasks[i].p);
          if (ok[c] && need[c] <= cap[c]) {
            treg[i] = rg[i];
            tclass[i] = rc[i];
            tres[i] = 1;
          }
        }
      }
      // simultaneous order: the coupling blocks to transform afterwards, one
      // per unordered pair of interfaces (p < q), each with workspace for
      // Y = A_pq Q_qc (|p| x |q| bound)
      struct SimEdge { int i, j; int32_t e; size_t y; };
      std::vector<SimEdge> sedges;
      if (sim) {
        std::vector<int> tix(n, -1);
        for (size_t i = 0; i < tasks.size(); ++i) tix[tasks[i].p] = (int)i;
        for (size_t i = 0; i < tasks.size(); ++i)
          for (int32_t e = tasks[i].nbeg; e < tasks[i].nend; ++e) {
            const int q = nbrs[e].q, j = tix[q];
            if (j < 0 || tasks[i].p >= q) continue;
            sedges.push_back({(int)i, j, e, wbytes});
            wbytes += align256((size_t)tasks[i].np * tasks[j].np * sizeof(T));
          }
      }
      if (!tasks.empty()) {
        char* wb = interp ? nullptr : (char*)h->scratch[(t + 1) & 1].ensure(wbytes);
        for (size_t i = 0; i < tasks.size() && wb; ++i) {
          tasks[i].V = (T*)(wb + woff[i].v);
          tasks[i].tau = (T*)(wb + woff[i].tau);
          tasks[i].Qc = (T*)(wb + woff[i].qc);
          tasks[i].gwork = (T*)(wb + woff[i].gw);
          cp_qc.push_back(tasks[i].Qc);
        }
        if (interp) {
          std::vector<int> tcol_(tasks.size());
          for (size_t i = 0; i < tasks.size(); ++i) tcol_[i] = colour_of(tasks[i].p);
          std::vector<int32_t> hsz = sz;
          interp_out = sparsify_interp<T>(h, tasks, tcol_, ncol, nbrs, hsz, d_cur, d_info + 2 * (L + 1) + t * maxcol,
                                          f_cls[t], eps, s);
        } else if (h->opts.compression == SPAND_RANDOMIZED) {
          cpqr_pid = h->prof.begin(F_CPQR, s);
          std::vector<int> tcolr(tasks.size());
          for (size_t i = 0; i < tasks.size(); ++i) tcolr[i] = colour_of(tasks[i].p);
          ell_fin = sparsify_randomized<T>(h, t, tasks, tcolr, ncol, nbrs, d_cur, eps, s);
          h->prof.end(cpqr_pid, s, 0.0, 0.0, 1);
        } else {
        // launch groups: (colour, cluster size)
        struct Group { int colour, C, res, G = 0; std::vector<int32_t> ids; size_t smem = 0; int maxm = 0; };
        // one pass: tasks bucketed by (colour, kernel, lane group, cluster
        // size, residency, CTAs per SM that their shared memory allows, 1-2):
        // a launch gives every CTA its group's largest need, so interfaces
        // with small chunks are not held to one CTA per SM by a few wide
        // ones; within a colour the register-resident groups come first
        std::map<std::tuple<int, int, int, int, int, int>, Group> buckets;
        for (size_t i = 0; i < tasks.size(); ++i) {
          const int c = colour_of(tasks[i].p), C = tclass[i], Gr = treg[i], res = tres[i];
          const int np_ = tasks[i].np, mm = tasks[i].m_max, nnb_ = tasks[i].nend - tasks[i].nbeg;
          size_t need;
          if (Gr) {
            need = cpqr_reg_smem<T>(Gr, nnb_, np_, (mm + C - 1) / C, C);
          } else {
            need = cq_fixed_smem<T>(nnb_, np_, (mm + C - 1) / C, C);
            if (res) need += (size_t)cq_ld<T>(np_) * ((mm + C - 1) / C) * sizeof(T);
          }
          // (at most two: the chunked kernel's registers hold two 256-thread CTAs per SM)
          const int per_sm = Gr ? 1 : (int)std::min<size_t>(2, std::max<size_t>(1, kSmemPerSM / (need + 1024)));
          Group& g = buckets[std::make_tuple(c, Gr ? 0 : 1, Gr, C, -res, -per_sm)];
          if (g.ids.empty()) {
            g.colour = c;
            g.C = C;
            g.res = res;
            g.G = Gr;
          }
          g.ids.push_back((int32_t)i);
          g.smem = std::max(g.smem, need);
          g.maxm = std::max(g.maxm, mm);
        }
        std::vector<Group> groups;
        groups.reserve(buckets.size());
        for (auto& kv : buckets) groups.push_back(std::move(kv.second));
        std::vector<int32_t> list;
        std::vector<size_t> gbeg;
        for (auto& g : groups) {
          gbeg.push_back(list.size());
          list.insert(list.end(), g.ids.begin(), g.ids.end());
        }
        Packer pk;
        size_t ot = pk.add(tasks), on = pk.add(nbrs), ol = pk.add(list);
        void* d = upload<T>(h, pk, s);
        ensure_streams(h);
        cpqr_pid = h->prof.begin(F_CPQR, s);
        size_t gi = 0;
        int64_t nformq = 0;  // k_form_q launches (one per colour)
        while (gi < groups.size()) {  // one colour at a time; its groups run side by side
          size_t ge = gi;
          while (ge < groups.size() && groups[ge].colour == groups[gi].colour) ++ge;
          CK(cudaEventRecord(h->ev_fork, s));
          for (size_t g = gi; g < ge; ++g) {
            cudaStream_t as = h->aux[(g - gi) % kAuxStreams];
            CK(cudaStreamWaitEvent(as, h->ev_fork, 0));
            const Group& G = groups[g];
            const size_t smem = G.smem;
            // 512 threads for one- and two-CTA interfaces (latency hiding)
            // when the launch fits in one wave; 256 for larger clusters
            // (cheaper block barriers) and for launches of more CTAs than
            // SMs (several CTAs per SM), unless the columns per CTA need 512
            const int cpg = (G.maxm + G.C - 1) / G.C;
            const bool one_wave = G.ids.size() * (size_t)G.C <= (size_t)num_sms();
            int nt = ((G.C <= 2 && one_wave) || cpg > CQ_CPT * 256) ? 512 : 256;
            // one wave with few columns per CTA, FP64: 512 threads in lane
            // groups of 2 or 4 per column, so that each step's column sweep
            // is shorter (measured at 64^3: FP64 form 350 -> 327 ms per step;
            // the FP32 sweeps are short enough that the extra threads and
            // shuffles cost more than they save, 18.5 -> 19.8 ms)
            int lg = 1;
            if (sizeof(T) == 8 && one_wave && cpg <= 256) {
              nt = 512;
              lg = cpg <= 128 ? 4 : 2;
            }
            const void* fn = cpqr_kernel<T>(G.res != 0, nt, lg);
            if (G.G) {
              nt = kCqrThreads;
              fn = cpqr_reg_kernel<T>(G.G);
            }
            ensure_smem(fn, smem);
            if (G.C > 8) ensure_nonportable_cluster(fn);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(G.ids.size() * G.C), 1, 1);
            cfg.blockDim = dim3((unsigned)nt, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = as;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)G.C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const CpqrTask<T>* a0 = at<const CpqrTask<T>>(d, ot);
            const int32_t* a1 = at<const int32_t>(d, ol) + gbeg[g];
            const CpqrNbr<T>* a2 = at<const CpqrNbr<T>>(d, on);
            T a4 = (T)eps;
            void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&d_cur, (void*)&a4};
            CK(cudaLaunchKernelExC(&cfg, fn, args));
            CK(cudaEventRecord(h->ev_join[(g - gi) % kAuxStreams], as));
          }
          for (size_t g = gi; g < std::min(ge, gi + (size_t)kAuxStreams); ++g)
            CK(cudaStreamWaitEvent(s, h->ev_join[(g - gi) % kAuxStreams], 0));
          // Q_pc of this colour's interfaces on the side stream, overlapping
          // the next colour's QR (nothing in the factorization reads Q_pc
          // before the compaction below)
          {
            constexpr int NTQ = 256, NWQ = NTQ / 32;
            const size_t l0 = gbeg[gi], l1 = ge < groups.size() ? gbeg[ge] : list.size();
            int kmx = 0;
            size_t need = 0;
            for (size_t li = l0; li < l1; ++li) {
              const CpqrTask<T>& tk = tasks[list[li]];
              const int km = std::min(tk.np, tk.m_max);
              kmx = std::max(kmx, km);
              need = std::max(need, align256((size_t)km * sizeof(T)) + (size_t)tk.np * km * sizeof(T));
            }
            const size_t qsm = std::min(need + 256, (size_t)227 * 1024);
            const int nb = std::max(1, (kmx + 2 * NWQ - 1) / (2 * NWQ));
            const void* fq = (const void*)k_form_q<T, NTQ>;
            ensure_smem(fq, qsm);
            CK(cudaEventRecord(h->ev_q, s));
            CK(cudaStreamWaitEvent(h->qs, h->ev_q, 0));
            const CpqrTask<T>* q0 = at<const CpqrTask<T>>(d, ot);
            const int32_t* q1 = at<const int32_t>(d, ol) + l0;
            const int q3 = nb, q4 = (int)(qsm / sizeof(T));
            void* qargs[] = {(void*)&q0, (void*)&q1, (void*)&d_cur, (void*)&q3, (void*)&q4};
            CK(cudaLaunchKernel(fq, dim3((unsigned)((l1 - l0) * nb)), dim3(NTQ), qargs, qsm, h->qs));
            ++nformq;
          }
          gi = ge;
        }
        CK(cudaEventRecord(h->ev_qdone, h->qs));
        CK(cudaStreamWaitEvent(s, h->ev_qdone, 0));
        int64_t nsim = 0;  // k_sim_gemm launches
        if (!sedges.empty()) {  // A_pq <- Q_pc^T (A_pq Q_qc): all reads in the first launch, all writes in the second
          std::vector<SimGemm<T>> g1, g2;
          std::vector<int32_t> o1{0}, o2{0};
          for (const SimEdge& se : sedges) {
            const CpqrTask<T>& tp = tasks[se.i];
            const CpqrTask<T>& tq = tasks[se.j];
            const CpqrNbr<T>& nb = nbrs[se.e];
            T* Y = (T*)(wb + se.y);
            T* Apq = tp.Rp + (size_t)nb.off_pq * tp.ldp;
            const int tm = (tp.np + SG_TM - 1) / SG_TM, tn = (tq.np + SG_TN - 1) / SG_TN;
            SimGemm<T> a{};  // Y (|p| x r_q) = A_pq Q_qc
            a.A = Apq;
            a.lda = tp.ldp;
            a.B = tq.Qc;
            a.ldb = tq.np;
            a.C = Y;
            a.ldc = tp.np;
            a.m = tp.np;
            a.n = tq.np;
            a.k = tq.np;
            a.mi = -1;
            a.ni = tq.p;
            a.tiles_m = tm;
            g1.push_back(a);
            o1.push_back(o1.back() + tm * tn);
            SimGemm<T> b{};  // X (r_p x r_q) = Q_pc^T Y into A_pq, X^T into A_qp
            b.A = tp.Qc;
            b.lda = tp.np;
            b.transA = 1;
            b.B = Y;
            b.ldb = tp.np;
            b.C = Apq;
            b.ldc = tp.ldp;
            b.C2 = nb.Rq + (size_t)nb.off_qp * nb.ldq;
            b.ldc2 = nb.ldq;
            b.m = tp.np;
            b.n = tq.np;
            b.k = tp.np;
            b.mi = tp.p;
            b.ni = tq.p;
            b.tiles_m = tm;
            g2.push_back(b);
            o2.push_back(o2.back() + tm * tn);
          }
          Packer pk2;
          const size_t a1 = pk2.add(g1), a2 = pk2.add(o1), a3 = pk2.add(g2), a4 = pk2.add(o2);
          void* d2 = upload<T>(h, pk2, s);
          const int nd = (int)sedges.size();
          k_sim_gemm<T><<<(unsigned)o1.back(), SG_NT, 0, s>>>(at<const SimGemm<T>>(d2, a1),
                                                              at<const int32_t>(d2, a2), nd, d_rank);
          CKLAUNCH();
          k_sim_gemm<T><<<(unsigned)o2.back(), SG_NT, 0, s>>>(at<const SimGemm<T>>(d2, a3),
                                                              at<const int32_t>(d2, a4), nd, d_rank);
          CKLAUNCH();
          nsim = 2;
        }
        if (sim) CK(cudaMemcpyAsync(d_cur, d_rank, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        h->prof.launches += (int64_t)groups.size() + nformq + nsim;
        h->prof.end(cpqr_pid, s, 0.0, 0.0, (int64_t)groups.size() + nformq + nsim);
        }
        build_elim_ops();  // host work overlapped with the sparsification kernels
        run_pending();
        int32_t* hcur = (int32_t*)h->stage.take((size_t)n * sizeof(int32_t));
        CK(cudaMemcpyAsync(hcur, d_cur, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::copy(hcur, hcur + n, sz_after.begin());
        h->stage.reset();  // every copy issued so far has executed
        for (size_t i = 0; i < tasks.size(); ++i) {
          const int rr = sz_after[tasks[i].p];
          if (rr == -2) throw Fail{SPAND_ERR_TIMEOUT, "sparsification: a cluster exchange timed out"};
          if (rr < 0) throw Fail{SPAND_ERR_STATE, "sparsification: launch shape refused by the kernel"};
        }
        check_pivots(t);
        for (const SimEdge& se : sedges) {  // algorithmic work of the two-sided transforms
          const double np_ = tasks[se.i].np, nq_ = tasks[se.j].np;
          const double rp = sz_after[tasks[se.i].p], rq = sz_after[tasks[se.j].p];
          const double fl = 2 * np_ * nq_ * rq + 2 * rp * np_ * rq;
          stt.factor_flops += fl;
          h->prof.add(cpqr_pid, fl, (np_ * nq_ + nq_ * rq + 2 * np_ * rq + np_ * rp + 2 * rp * rq) * sizeof(T));
        }
      }
      for (int sidx : seps) sz_after[sidx] = 0;
      // compact Q_pc (|p| x r) into the factor
      std::vector<CopyTask<T>> qcopy;
      std::vector<int> sq_of(n, -1);
      for (size_t i = 0; i < sq_cluster.size(); ++i) sq_of[sq_cluster[i]] = (int)i;
      for (size_t i = 0; i < cp_cluster.size() && !interp; ++i) {
        const int p = cp_cluster[i];
        const int r = sz_after[p];
        // sparsified: Q_pc (|p| x r); r = 0 keeps a non-null empty basis
        T* Q = (T*)h->persist.alloc((size_t)sz[p] * std::max(r, 1) * sizeof(T));
        if (r > 0) qcopy.push_back({cp_qc[i], Q, sz[p], sz[p], sz[p], r, 0, 0});
        SqOp<T>& so = sqops[sq_of[p]];
        so.Q = Q;
        so.r = r;
        const double np_ = sz[p], m = lay.W[p] - sz[p], rr = r;
        // CPQR of A_pn to rank r; randomized: sketch and projection (2 np m ell
        // each) and the QR of the np x ell sketch
        const double el = i < ell_fin.size() ? ell_fin[i] : 0.0;
        const double qfl = ell_fin.empty() ? 4 * np_ * m * rr - 2 * rr * rr * (np_ + m) + 4 * rr * rr * rr / 3
                                           : 4 * np_ * m * el + 4 * np_ * el * el - 4 * el * el * el / 3;
        stt.factor_flops += qfl;
        // algorithmic bytes: A_pn read once, W written twice, Q_pc written
        h->prof.add(cpqr_pid, qfl, (np_ * m + 2 * rr * m + np_ * rr) * sizeof(T));
        stt.mem_f += (int64_t)sz[p] * r;
      }
      for (auto& so : sqops) sm_r = std::max(sm_r, (size_t)std::max(so.r, 1) * sizeof(double));
      copy_batch<T>(h, qcopy, s);
      if (interp) {
        // apply groups of the step's interpolative transforms: T_p (U = I,
        // X^T = T_cf, c against f), then the elimination of f against c; p
        // keeps the slots of c, in pivot order
        std::vector<ElimSpec<T>> tsp, fsp;
        for (const InterpOut<T>& o : interp_out) {
          if (o.p < 0) continue;
          const std::vector<int32_t>& sl = slots[o.p];
          std::vector<int32_t> cs(o.r), fs(o.nf);
          for (int a = 0; a < o.r; ++a) cs[a] = sl[o.perm[a]];
          for (int j = 0; j < o.nf; ++j) fs[j] = sl[o.perm[o.r + j]];
          if (o.nf > 0) {
            if (o.r > 0) tsp.push_back({o.XT, nullptr, o.r, cs, fs});
            fsp.push_back({o.F + (size_t)o.ldf * o.nf, o.Yf, o.ldf, fs, cs});
          }
          kept_slots[o.p] = std::move(cs);
          has_kept[o.p] = 1;
        }
        interp_steps.push_back(make_elim_step<T>(h, tsp, s));
        interp_steps.push_back(make_elim_step<T>(h, fsp, s));
      }
    } else {
      CK(cudaEventRecord(tm.at(t, 2), s));
    }
    CK(cudaEventRecord(tm.at(t, 3), s));
    if (!elim_ops_built) build_elim_ops();
    h->sizes_after[t - 1] = sz_after;
    // ------------------------------------------------ merge (Sec. 2.7)
    Layout<T> nxt;
    if (t < L) {
      const StepStruct& ns = tr.steps[t];
      std::vector<int32_t> nsz(ns.n, 0), pof(n, -1), ro(n, 0);
      std::vector<std::vector<int32_t>> nslots(ns.n);
      for (int P = 0; P < ns.n; ++P) {
        int32_t o = 0;
        for (int32_t e = ns.child_ptr[P]; e < ns.child_ptr[P + 1]; ++e) {
          const int32_t a = ns.child_idx[e];
          pof[a] = P;
          ro[a] = o;
          o += sz_after[a];
          const std::vector<int32_t>& ks = has_kept[a] ? kept_slots[a] : slots[a];
          nslots[P].insert(nslots[P].end(), ks.begin(), ks.begin() + sz_after[a]);
        }
        nsz[P] = o;
      }
      nxt = make_layout<T>(h, t + 1, nsz, s);
      if (h->mplan.size() < (size_t)L + 1) h->mplan.resize((size_t)L + 1);
      auto& mp = h->mplan[t];
      if (!mp.built) {
        mp.ptr.assign(1, 0);
        for (int a : rems) {
          const int P = pof[a];
          auto add = [&](int b, int32_t e) {
            const int Q = pof[b];
            int32_t tg = -1;
            if (Q != P) {
              tg = nxt.edge_of(P, Q);
              if (tg < 0) tg = -2;
            }
            mp.b.push_back(b);
            mp.src.push_back(e);
            mp.tgt.push_back(tg);
          };
          add(a, -1);
          for (int32_t e = lay.nptr[a]; e < lay.nptr[a + 1]; ++e) add(lay.nidx[e], e);
          mp.ptr.push_back((int32_t)mp.b.size());
        }
        mp.built = true;
      }
      std::vector<CopyTask<T>> cps;
      cps.reserve(mp.b.size());
      for (size_t ia = 0; ia < rems.size(); ++ia) {
        const int a = rems[ia];
        if (sz_after[a] <= 0) continue;
        const int P = pof[a];
        T* const dst0 = nxt.row[P] + ro[a];
        for (int32_t k = mp.ptr[ia]; k < mp.ptr[ia + 1]; ++k) {
          const int b = mp.b[k], tg = mp.tgt[k];
          if (sz_after[b] <= 0 || tg == -2) continue;
          const int32_t tc = (tg < 0 ? 0 : nxt.noff[tg]) + ro[b];
          const int32_t src_col = mp.src[k] < 0 ? 0 : lay.noff[mp.src[k]];
          CopyTask<T> c;
          c.src = lay.row[a] + (size_t)src_col * lay.ld[a];
          c.dst = dst0 + (size_t)tc * nxt.ld[P];
          c.lds = lay.ld[a];
          c.ldd = nxt.ld[P];
          c.rows = sz_after[a];
          c.cols = sz_after[b];
          c.trans = 0;
          c.pad = 0;
          cps.push_back(c);
        }
      }
      copy_batch<T>(h, cps, s);
      sz = nsz;
      slots_of_step = std::move(slots);
      slots = std::move(nslots);
    } else {
      slots_of_step = std::move(slots);
    }
    CK(cudaEventRecord(tm.at(t, 4), s));
    run_pending();  // the previous step's program, if the GPU never waited for us
    // The step's apply program (scaling + coarse-basis ops, upload) is built
    // later, during the next step's sparsification kernels (run_pending), so
    // that the rank-dependent GPU work (merge, next elimination) is issued
    // first.  Steps are finalized in order.
    {
      std::vector<std::vector<int32_t>> prev_slots = std::move(slots_of_step);
      pending = [h, s, &apply, prev_slots = std::move(prev_slots), ap = std::move(ap), eops = std::move(eops),
                 sqops = std::move(sqops), sq_cluster = std::move(sq_cluster), aslots = std::move(aslots),
                 tslot = std::move(tslot), tptr = std::move(tptr), tidx = std::move(tidx), it_fy = std::move(it_fy),
                 it_fu = std::move(it_fu), it_ba = std::move(it_ba), it_bx = std::move(it_bx), nassign, sm_ns, sm_m,
                 sm_np, sm_r, tmp_off, interp_steps = std::move(interp_steps)]() mutable {
      // slots, save areas, temporaries and work items of the scaling +
      // coarse-basis ops (step-t slot lists)
      std::vector<ApplyItem> it_sy = h->poolitem.take(), it_sc = h->poolitem.take(), it_sz = h->poolitem.take(),
                             it_sx = h->poolitem.take();
      {
        int64_t save = h->save_len;
        for (size_t i = 0; i < sqops.size(); ++i) {
          SqOp<T>& so = sqops[i];
          const int p = sq_cluster[i];
          so.slot = (int64_t)aslots.size();
          aslots.insert(aslots.end(), prev_slots[p].begin(), prev_slots[p].end());
          so.save = save;
          save += so.np + so.r;
          so.tz = tmp_off;
          tmp_off += so.np;
          const int32_t op = (int32_t)i;
          for (int32_t r0 = 0; r0 < so.np; r0 += RB) {
            it_sy.push_back({op, r0});
            it_sz.push_back({op, r0});
          }
          for (int32_t c0 = 0; c0 < so.r; c0 += AP_COLS) it_sc.push_back({op, c0});
          for (int32_t c0 = 0; c0 < so.np; c0 += AP_COLS) it_sx.push_back({op, c0});
        }
        h->save_len = save;
        h->tmp_len = std::max(h->tmp_len, tmp_off);
      }
      {  // upload the step's apply program
        Packer pk;
        size_t oe = pk.add(eops), os = pk.add(sqops), osl = pk.add(aslots);
        size_t osy = pk.add(it_sy), osc = pk.add(it_sc), osz = pk.add(it_sz), osx = pk.add(it_sx);
        size_t ots = pk.add(tslot), otp = pk.add(tptr), oti = pk.add(tidx);
        size_t ofy = pk.add(it_fy), ofu = pk.add(it_fu), oba = pk.add(it_ba), obx = pk.add(it_bx);
        void* d = nullptr;
        if (!pk.empty()) {
          d = h->persist.alloc(pk.size);
          void* src = h->stage.take(pk.size);
          pk.write(src);
          CK(cudaMemcpyAsync(d, src, pk.size, cudaMemcpyHostToDevice, s));
        }
        ap.n_elim = (int)eops.size();
        ap.n_sq = (int)sqops.size();
        ap.elim = at<const ElimOp<T>>(d, oe);
        ap.sq = at<const SqOp<T>>(d, os);
        ap.n_sy = (int)it_sy.size();
        ap.n_sc = (int)it_sc.size();
        ap.n_sz = (int)it_sz.size();
        ap.n_sx = (int)it_sx.size();
        ap.sy = at<const ApplyItem>(d, osy);
        ap.sc = at<const ApplyItem>(d, osc);
        ap.sz = at<const ApplyItem>(d, osz);
        ap.sx = at<const ApplyItem>(d, osx);
        ap.slots = at<const int32_t>(d, osl);
        ap.ntgt = (int64_t)tslot.size();
        ap.nassign = nassign;
        ap.tslot = at<const int32_t>(d, ots);
        ap.tptr = at<const int64_t>(d, otp);
        ap.tidx = at<const int64_t>(d, oti);
        ap.n_fy = (int)it_fy.size();
        ap.n_fu = (int)it_fu.size();
        ap.n_ba = (int)it_ba.size();
        ap.n_bx = (int)it_bx.size();
        ap.fy = at<const ApplyItem>(d, ofy);
        ap.fu = at<const ApplyItem>(d, ofu);
        ap.ba = at<const ApplyItem>(d, oba);
        ap.bx = at<const ApplyItem>(d, obx);
        ap.sm_ns = sm_ns;
        ap.sm_m = sm_m;
        ap.sm_np = sm_np;
        ap.sm_r = sm_r;
        apply.push_back(ap);
        for (const ApplyStep<T>& x : interp_steps)
          if (x.n_elim) apply.push_back(x);
      }
      // the host arrays have been copied to pinned staging: back to the pools
      h->pool32.give(std::move(aslots));
      h->pool32.give(std::move(tslot));
      h->pool64.give(std::move(tptr));
      h->pool64.give(std::move(tidx));
      for (auto* v : {&it_fy, &it_fu, &it_ba, &it_bx, &it_sy, &it_sc, &it_sz, &it_sx}) h->poolitem.give(std::move(*v));
      };
    }

    if (t < L) lay = std::move(nxt);
  }
  run_pending();
  CK(cudaStreamSynchronize(s));
  check_pivots(L);
  {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, tm.at(0, 0), tm.at(0, 1)));
    h->phase_ms[3] += ms;
    for (int t = 1; t <= L; ++t)
      for (int k = 0; k < 4; ++k) {
        CK(cudaEventElapsedTime(&ms, tm.at(t, k), tm.at(t, k + 1)));
        h->phase_ms[k] += ms;
      }
  }
  build_apply_program<T>(h, apply, s);
  if constexpr (std::is_same<T, double>::value) {
    h->apply64 = std::move(apply);
    h->apply32.clear();
  } else {
    h->apply32 = std::move(apply);
    h->apply64.clear();
  }
  return SPAND_OK;
}

// ---------------------------------------------------------------- apply / PCG

// tmp: h->tmp_len doubles of per-step temporaries; save: h->save_len doubles
// of sparsification forward inputs (both scratch; nothing needs to start at 0).
// One cooperative launch runs the whole apply program; a barrier timeout is
// recorded in d_bar[1] and reported by check_apply().
template <typename TF>
static void apply_prec(spand_handle h, double* x, double* tmp, double* save, cudaStream_t s) {
  if (!h->n_aprog) return;
  const int pid = h->prof.begin(F_APPLY, s);
  unsigned* bar = (unsigned*)h->d_bar.p;
  int* err = (int*)(bar + 1);
  CK(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
  const ApplyPhase<TF>* ph = (const ApplyPhase<TF>*)h->aprog;
  int nph = h->n_aprog;
  unsigned lim = h->apply_spin_limit, bias = h->apply_bias;
  void* args[] = {(void*)&ph, (void*)&nph, (void*)&x,   (void*)&tmp, (void*)&save,
                  (void*)&bar, (void*)&err, (void*)&lim, (void*)&bias};
  CK(cudaLaunchCooperativeKernel((const void*)k_apply<TF>, dim3((unsigned)h->apply_grid), dim3(AT), args,
                                 h->apply_smem, s));
  CKLAUNCH();
  h->prof.launches += 1;
  h->prof.end(pid, s, 0.0, h->st.apply_bytes, 1);
}

static void apply_any(spand_handle h, double* x, double* tmp, double* save, cudaStream_t s) {
  if (h->fprec == SPAND_FP64) apply_prec<double>(h, x, tmp, save, s);
  else apply_prec<float>(h, x, tmp, save, s);
}

// Reads (after the stream has been synchronised) and clears the apply's
// barrier-timeout flag.
static void check_apply(spand_handle h) {
  if (!h->d_bar.p) return;
  int flag = 0;
  CK(cudaMemcpy(&flag, (unsigned*)h->d_bar.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemset((unsigned*)h->d_bar.p + 1, 0, sizeof(int)));
    throw Fail{SPAND_ERR_TIMEOUT, "preconditioner apply: a grid barrier timed out"};
  }
}

static void apply_any(spand_handle h, double* x, cudaStream_t s) {
  apply_any(h, x, (double*)h->d_tmp.p, (double*)h->d_save.p, s);
}

// Tile-shape autotuner of the apply (the grid of its cooperative launch):
// the first apply after a handle's first factorization times 1 .. 4 CTAs per
// SM (two applications each, on a scratch vector) and keeps the fastest for
// the handle's later factorizations and solves.  Every item of a phase is
// computed by one CTA in a fixed order whatever the grid, so the choice never
// changes a bit of z.  More CTAs stream the large leaf phases faster; fewer
// make the grid barriers of many small phases cheaper.
static void apply_autotune(spand_handle h, double* scratch, cudaStream_t s) {
  if (h->apply_ctas > 0 || !h->n_aprog) return;
  int nsm = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaMemsetAsync(scratch, 0, (size_t)h->n * sizeof(double), s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = h->prof.on;
  h->prof.on = false;
  float best = 0.f;
  int pick = h->apply_per_sm_max;
  for (int c = 1; c <= h->apply_per_sm_max; ++c) {
    h->apply_grid = nsm * c;
    apply_any(h, scratch, s);  // warm-up
    CK(cudaEventRecord(e0, s));
    apply_any(h, scratch, s);
    apply_any(h, scratch, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (c == 1 || ms < best) best = ms, pick = c;
  }
  h->prof.on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->apply_ctas = pick;
  h->apply_grid = nsm * pick;
}

static void ensure_solve_buffers(spand_handle h) {
  const int64_t n = std::max<int64_t>(h->n, 1);
  h->d_vec.ensure((size_t)(7 * n + RED_BLOCKS + 16) * sizeof(double));
  h->d_tmp.ensure((size_t)std::max<int64_t>(h->tmp_len, 1) * sizeof(double));
  h->d_save.ensure((size_t)std::max<int64_t>(h->save_len, 1) * sizeof(double));
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace spand

// ==================================================================== C ABI

#define API_BEGIN try {
#define API_END                                              \
  }                                                          \
  catch (const Fail& f) {                                    \
    g_err = f.msg;                                           \
    return f.code;                                           \
  }                                                          \
  catch (const std::bad_alloc&) {                            \
    g_err = "host allocation failed";                        \
    return SPAND_ERR_OOM;                                    \
  }                                                          \
  catch (const std::exception& e) {                          \
    g_err = e.what();                                        \
    return SPAND_ERR_INVALID_ARG;                            \
  }                                                          \
  catch (...) {                                              \
    g_err = "unknown error";                                 \
    return SPAND_ERR_INVALID_ARG;                            \
  }

extern "C" {

void spand_default_opts(spand_opts* o) {
  if (!o) return;
  o->levels = 8;
  o->eps = 1e-2;
  o->skip = 0;
  o->precision = SPAND_FP64;
  o->maxit = 500;
  o->tol = 1e-10;
  o->sparsify_order = SPAND_COLOURED;
  o->compression = SPAND_CPQR;
  o->sketch_seed = 0;
  o->variant = SPAND_ORTHS;
}

const char* spand_error_string(int code) {
  switch (code) {
    case SPAND_OK: return "ok";
    case SPAND_ERR_INVALID_ARG: return "invalid argument";
    case SPAND_ERR_NOT_SPD: return "matrix (or a pivot block) is not positive definite";
    case SPAND_ERR_NO_CONVERGENCE: return "PCG did not converge within maxit";
    case SPAND_ERR_CUDA: return "CUDA error";
    case SPAND_ERR_OOM: return "out of memory";
    case SPAND_ERR_STATE: return "call out of order";
    case SPAND_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    default: return "unknown error code";
  }
}

const char* spand_last_error(void) { return g_err.c_str(); }

int spand_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals, const double* coords,
                  int32_t dim, const spand_opts* opts, spand_handle* out) {
  if (!out) { g_err = "out is NULL"; return SPAND_ERR_INVALID_ARG; }
  *out = nullptr;
  API_BEGIN
  g_err.clear();
  if (!opts) throw Fail{SPAND_ERR_INVALID_ARG, "opts is NULL"};
  if (opts->levels < 1 || opts->levels > 30) throw Fail{SPAND_ERR_INVALID_ARG, "levels must be in [1, 30]"};
  if (!(opts->eps >= 0.0)) throw Fail{SPAND_ERR_INVALID_ARG, "eps must be >= 0"};
  if (opts->skip < 0) throw Fail{SPAND_ERR_INVALID_ARG, "skip must be >= 0"};
  if (opts->precision != SPAND_FP64 && opts->precision != SPAND_FP32 && opts->precision != SPAND_TF32 &&
      opts->precision != SPAND_BF16)
    throw Fail{SPAND_ERR_INVALID_ARG, "unknown precision"};
  if (opts->maxit < 1 || !(opts->tol > 0.0)) throw Fail{SPAND_ERR_INVALID_ARG, "maxit >= 1 and tol > 0 required"};
  if (opts->sparsify_order != SPAND_COLOURED && opts->sparsify_order != SPAND_SIMULTANEOUS)
    throw Fail{SPAND_ERR_INVALID_ARG, "unknown sparsify_order"};
  if (opts->compression != SPAND_CPQR && opts->compression != SPAND_RANDOMIZED)
    throw Fail{SPAND_ERR_INVALID_ARG, "unknown compression"};
  if (opts->compression == SPAND_RANDOMIZED && opts->sparsify_order != SPAND_COLOURED)
    throw Fail{SPAND_ERR_INVALID_ARG, "randomized compression runs in the coloured order only"};
  if (opts->variant != SPAND_ORTHS && opts->variant != SPAND_INS && opts->variant != SPAND_IN)
    throw Fail{SPAND_ERR_INVALID_ARG, "unknown variant"};
  if (opts->variant != SPAND_ORTHS &&
      (opts->sparsify_order != SPAND_COLOURED || opts->compression != SPAND_CPQR))
    throw Fail{SPAND_ERR_INVALID_ARG, "the interpolative variants need the coloured order and column-pivoted QR"};
  if (n > INT32_MAX - 1) throw Fail{SPAND_ERR_INVALID_ARG, "n too large"};
  if (coords && (dim < 1 || dim > 8)) throw Fail{SPAND_ERR_INVALID_ARG, "dim must be in [1, 8]"};
  std::string err;
  if (validate_csr(n, rowptr, colind, err)) throw Fail{SPAND_ERR_INVALID_ARG, err};
  const int64_t nnz = n ? rowptr[n] : 0;
  if (nnz && !vals) throw Fail{SPAND_ERR_INVALID_ARG, "vals is NULL"};
  auto t0 = std::chrono::steady_clock::now();
  std::unique_ptr<spand_handle_s> h(new spand_handle_s());
  h->opts = *opts;
  h->n = n;
  h->nnz = nnz;
  h->rowptr.assign(rowptr, rowptr + n + 1);
  h->colind.assign(colind, colind + nnz);
  h->vals.assign(vals, vals + nnz);
  if (analyze_tree(n, rowptr, colind, coords, dim, opts->levels, h->tree, err))
    throw Fail{SPAND_ERR_INVALID_ARG, err};
  const Tree& tr = h->tree;
  // position of every vertex, its cluster and local index
  std::vector<int32_t> pos(n), cl(n), loc(n);
  for (int64_t i = 0; i < n; ++i) pos[tr.perm[i]] = (int32_t)i;
  const int nc = (int)tr.cluster_ptr.size() - 1;
  for (int c = 0; c < nc; ++c)
    for (int32_t i = tr.cluster_ptr[c]; i < tr.cluster_ptr[c + 1]; ++i) {
      cl[tr.perm[i]] = c;
      loc[tr.perm[i]] = i - tr.cluster_ptr[c];
    }
  // step-1 assembly map (same row layout rule as the factorization)
  const StepStruct& s1 = tr.steps.empty() ? StepStruct() : tr.steps[0];
  h->asm_row.assign(nnz, -1);
  h->asm_off.assign(nnz, 0);
  if (n > 0) {
    std::vector<int32_t> csz(nc);
    for (int c = 0; c < nc; ++c) csz[c] = tr.cluster_ptr[c + 1] - tr.cluster_ptr[c];
    std::vector<std::vector<std::pair<int32_t, int32_t>>> coff(nc);  // (neighbour, col offset)
    for (int c = 0; c < nc; ++c) {
      const bool el = s1.elim[c];
      const int32_t b = el ? s1.adj_ptr[c] : s1.adjf_ptr[c];
      const int32_t e = el ? s1.adj_ptr[c + 1] : s1.adjf_ptr[c + 1];
      int32_t w = csz[c];
      for (int32_t k = b; k < e; ++k) {
        const int32_t q = el ? s1.adj_idx[k] : s1.adjf_idx[k];
        coff[c].push_back({q, w});
        w += csz[q];
      }
    }
    for (int64_t v = 0; v < n; ++v)
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        const int32_t w = colind[e];
        const int32_t ci = cl[v], cj = cl[w];
        int32_t col = -1;
        if (ci == cj) col = 0;
        else {
          auto& l = coff[ci];
          auto it = std::lower_bound(l.begin(), l.end(), std::make_pair(cj, INT32_MIN));
          if (it != l.end() && it->first == cj) col = it->second;
        }
        if (col < 0) continue;  // entry (n, s) of an eliminated s: held in s's row only
        const int64_t ld = row_ld(csz[ci]);
        h->asm_row[e] = ci;
        h->asm_off[e] = loc[v] + (int64_t)(col + loc[w]) * ld;
      }
  }
  // Envelope of every step-1 pivot block (the rows of A within one cluster
  // eliminated first, in cluster order): f(i) = the first row holding a
  // nonzero of column i.  U keeps that envelope, so tiles further than
  // bw = max_i (i/64 - f(i)/64) above the diagonal stay zero; the row lengths
  // r_j = #{i >= j : f(i) <= j} of U give the Cholesky flops sum_j r_j^2.
  h->env_bw.assign(nc, 0);
  h->env_bw32.assign(nc, 0);
  h->env_band.assign(nc, 0);
  h->env_flops.assign(nc, 0.0);
  h->env_nnz.assign(nc, 0.0);
  if (n > 0) {
    std::vector<int32_t> f;
    std::vector<int64_t> cnt;
    for (int c = 0; c < nc; ++c) {
      if (!s1.elim[c]) continue;
      const int32_t b = tr.cluster_ptr[c], sz = tr.cluster_ptr[c + 1] - b;
      f.resize(sz);
      for (int32_t i = 0; i < sz; ++i) {
        const int32_t v = tr.perm[b + i];
        int32_t fi = i;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
          const int32_t w = colind[e];
          if (cl[w] == c && loc[w] < fi) fi = loc[w];
        }
        f[i] = fi;
      }
      int32_t bw = 0, bw32 = 0, band = 0;
      double nnzU = 0;
      cnt.assign((size_t)sz + 1, 0);
      for (int32_t i = 0; i < sz; ++i) {
        bw = std::max(bw, i / 64 - f[i] / 64);
        bw32 = std::max(bw32, i / 32 - f[i] / 32);
        band = std::max(band, i - f[i]);
        nnzU += i - f[i] + 1;
        ++cnt[f[i]];  // column i covers rows f(i) .. i
        --cnt[i + 1];
      }
      double fl = 0, r = 0;
      for (int32_t j = 0; j < sz; ++j) {
        r += (double)cnt[j];
        fl += r * r;
      }
      const int32_t ntile = (sz + 63) / 64, ntile32 = (sz + 31) / 32;
      h->env_bw[c] = (bw + 1 >= ntile) ? 0 : bw;  // 0: dense (no tile is structurally zero)
      h->env_bw32[c] = (bw32 + 1 >= ntile32) ? 0 : bw32;
      h->env_band[c] = (band + 1 >= sz) ? 0 : band;
      h->env_flops[c] = fl;
      h->env_nnz[c] = nnzU;
    }
  }
  // A in cluster order
  h->prow.assign(n + 1, 0);
  h->pcol.resize(nnz);
  h->pval_src.resize(nnz);
  {
    std::vector<std::pair<int32_t, int64_t>> rowbuf;
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int32_t v = tr.perm[i];
      rowbuf.clear();
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) rowbuf.push_back({pos[colind[e]], e});
      std::sort(rowbuf.begin(), rowbuf.end());
      for (auto& pr : rowbuf) {
        h->pcol[o] = pr.first;
        h->pval_src[o] = pr.second;
        ++o;
      }
      h->prow[i + 1] = o;
    }
  }
  h->st.t_analyze_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return SPAND_OK;
  API_END
}

int spand_factorize(spand_handle h, const double* vals, void* cuda_stream) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  API_BEGIN
  g_err.clear();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto t0 = std::chrono::steady_clock::now();
  h->factored = false;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (h->device >= 0 && h->device != dev) throw Fail{SPAND_ERR_STATE, "handle was factorized on another device"};
  h->device = dev;
  const int64_t n = h->n, nnz = h->nnz;
  if (!h->consts_ready) {
    h->d_asm_row.ensure(std::max<int64_t>(nnz, 1) * sizeof(int32_t));
    h->d_asm_off.ensure(std::max<int64_t>(nnz, 1) * sizeof(int64_t));
    h->d_prow.ensure((n + 1) * sizeof(int64_t));
    h->d_pcol.ensure(std::max<int64_t>(nnz, 1) * sizeof(int32_t));
    h->d_pval_src.ensure(std::max<int64_t>(nnz, 1) * sizeof(int64_t));
    h->d_perm.ensure(std::max<int64_t>(n, 1) * sizeof(int32_t));
    if (nnz) {
      CK(cudaMemcpy(h->d_asm_row.p, h->asm_row.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_asm_off.p, h->asm_off.data(), nnz * sizeof(int64_t), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_pcol.p, h->pcol.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_pval_src.p, h->pval_src.data(), nnz * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(h->d_prow.p, h->prow.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (n) CK(cudaMemcpy(h->d_perm.p, h->tree.perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    h->consts_ready = true;
  }
  h->d_vals.ensure(std::max<int64_t>(nnz, 1) * sizeof(double));
  h->d_pval.ensure(std::max<int64_t>(nnz, 1) * sizeof(double));
  if (nnz) {
    const double* src = vals ? vals : h->vals.data();
    const bool dsrc = vals && is_device_ptr(vals);
    CK(cudaMemcpyAsync(h->d_vals.p, src, nnz * sizeof(double), dsrc ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (vals && !dsrc) std::memcpy(h->vals.data(), vals, nnz * sizeof(double));
    // permuted values for the SpMV: pval[k] = vals[pval_src[k]]
    k_gather_vals<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 4096), 256, 0, s>>>(
        nnz, (const int64_t*)h->d_pval_src.p, (const double*)h->d_vals.p, (double*)h->d_pval.p);
    CKLAUNCH();
    h->prof.launches += 1;
  }
  h->tmp_len = 0;
  h->save_len = 0;
  int rc;
  if (n == 0) {  // empty system: an empty factorization (apply and solve return at once)
    h->sizes_before.assign(h->tree.L, {});
    h->sizes_after.assign(h->tree.L, {});
    for (double& v : h->phase_ms) v = 0;
    h->st.size_top = 0;
    h->st.mem_f = 0;
    h->st.factor_flops = 0;
    h->st.fail_step = 0;
    h->st.fail_cluster = -1;
    rc = SPAND_OK;
  } else if (h->opts.precision == SPAND_FP64) {
    rc = factorize_impl<double>(h, s);
  } else {
    rc = factorize_impl<float>(h, s);
  }
  h->fprec = h->opts.precision;
  CK(cudaStreamSynchronize(s));
  h->st.t_factor_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  h->st.device_bytes = (int64_t)(h->persist.bytes_held + h->descs.bytes_held + h->scratch[0].cap + h->scratch[1].cap +
                                   h->d_piv64.cap);
  const size_t esz = h->fprec == SPAND_FP64 ? 8 : 4;
  h->st.apply_bytes = 2.0 * (double)h->st.mem_f * esz;
  h->factored = rc == SPAND_OK;
  return rc;
  API_END
}


int spand_apply(spand_handle h, const double* r_dev, double* z_dev, void* cuda_stream) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  API_BEGIN
  g_err.clear();
  if (!h->factored) throw Fail{SPAND_ERR_STATE, "spand_apply before a successful spand_factorize"};
  if (h->n && (!r_dev || !z_dev)) throw Fail{SPAND_ERR_INVALID_ARG, "null vector"};
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ensure_solve_buffers(h);
  const int64_t n = h->n;
  if (n == 0) return SPAND_OK;
  double* w = (double*)h->d_vec.p;
  apply_autotune(h, w, s);
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_permute<<<g, 256, 0, s>>>(n, (const int32_t*)h->d_perm.p, r_dev, w, 1);
  CKLAUNCH();
  apply_any(h, w, s);
  k_permute<<<g, 256, 0, s>>>(n, (const int32_t*)h->d_perm.p, w, z_dev, 0);
  CKLAUNCH();
  h->prof.launches += 2;
  CK(cudaStreamSynchronize(s));
  check_apply(h);
  return SPAND_OK;
  API_END
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free apply
//
// spand_apply allocates its work vectors (device memory) on first use.  Some
// callers cannot allow that: code that runs while another component owns the
// whole device memory pool (a framework's caching allocator with a fixed
// budget), or a latency-critical loop where cudaMalloc / cudaFree would add
// their implicit device-wide synchronisation.  spand_apply_noalloc computes the
// same z = M M^T r with its work vectors in one fixed array that lives in the
// library image itself (a static __device__ array, kNoAllocMaxDoubles doubles =
// 16 MiB, resident on every GPU that loads the library until the process
// exits), so the call itself never allocates.
namespace spand {
constexpr int64_t kNoAllocMaxDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxDoubles];
constexpr int kNoAllocMaxDevices = 64;
// device address of the array, per device (looked up once; threads that race
// on the first call store the same value)
static std::atomic<double*> g_noalloc_addr[kNoAllocMaxDevices];
}  // namespace spand

extern "C" {

int spand_apply_noalloc(spand_handle h, const double* r_dev, double* z_dev, void* cuda_stream) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  API_BEGIN
  g_err.clear();
  if (!h->factored) throw Fail{SPAND_ERR_STATE, "spand_apply_noalloc before a successful spand_factorize"};
  if (h->n && (!r_dev || !z_dev)) throw Fail{SPAND_ERR_INVALID_ARG, "null vector"};
  const int64_t n = h->n;
  const int64_t need = n + std::max<int64_t>(h->tmp_len, 0) + std::max<int64_t>(h->save_len, 0);
  if (need > kNoAllocMaxDoubles)
    throw Fail{SPAND_ERR_INVALID_ARG, "spand_apply_noalloc: this factorization needs " + std::to_string(need) +
                                          " doubles of work space, the fixed array holds " +
                                          std::to_string(kNoAllocMaxDoubles)};
  if (n == 0) return SPAND_OK;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != h->device)
    throw Fail{SPAND_ERR_INVALID_ARG, "spand_apply_noalloc: the current device is not the one the handle was "
                                      "factorized on"};
  if (dev < 0 || dev >= kNoAllocMaxDevices) throw Fail{SPAND_ERR_INVALID_ARG, "device ordinal out of range"};
  double* w = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!w) {  // once per device, with that device current
    CK(cudaGetSymbolAddress((void**)&w, g_noalloc_scratch));
    g_noalloc_addr[dev].store(w, std::memory_order_release);
  }
  double* tmp = w + n;
  double* save = tmp + h->tmp_len;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_permute<<<g, 256, 0, s>>>(n, (const int32_t*)h->d_perm.p, r_dev, w, 1);
  CKLAUNCH();
  apply_any(h, w, tmp, save, s);
  k_permute<<<g, 256, 0, s>>>(n, (const int32_t*)h->d_perm.p, w, z_dev, 0);
  CKLAUNCH();
  h->prof.launches += 2;
  CK(cudaStreamSynchronize(s));
  check_apply(h);
  return SPAND_OK;
  API_END
}

int spand_solve(spand_handle h, const double* b, double* x, int32_t* iters, double* relres, void* cuda_stream) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  API_BEGIN
  g_err.clear();
  if (!h->factored) throw Fail{SPAND_ERR_STATE, "spand_solve before a successful spand_factorize"};
  const int64_t n = h->n;
  if (n && (!b || !x)) throw Fail{SPAND_ERR_INVALID_ARG, "null vector"};
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto t0 = std::chrono::steady_clock::now();
  ensure_solve_buffers(h);
  if (n == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return SPAND_OK;
  }
  double* V = (double*)h->d_vec.p;
  double *bp = V, *xv = V + n, *r = V + 2 * n, *z = V + 3 * n, *p = V + 4 * n, *q = V + 5 * n, *io = V + 6 * n;
  apply_autotune(h, z, s);
  double* part = V + 7 * n;
  double* sc = part + RED_BLOCKS;  // scalars
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  CK(cudaMemcpyAsync(io, b, n * sizeof(double), bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  const int32_t* perm = (const int32_t*)h->d_perm.p;
  const int64_t* rp = (const int64_t*)h->d_prow.p;
  const int32_t* ci = (const int32_t*)h->d_pcol.p;
  const double* va = (const double*)h->d_pval.p;
  k_permute<<<g, 256, 0, s>>>(n, perm, io, bp, 1);
  CKLAUNCH();
  h->prof.launches += 1;
  CK(cudaMemsetAsync(xv, 0, n * sizeof(double), s));
  auto dot = [&](const double* a, const double* c, double* out) {
    k_dot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, c, part);
    CKLAUNCH();
    k_reduce<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, out);
    CKLAUNCH();
    h->prof.launches += 2;
  };
  auto read = [&](const double* d) {
    double v = 0;
    CK(cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->prof.flush();
    return v;
  };
  const double pcg_bytes = (double)h->nnz * 12 + (double)(n + 1) * 8 + 9.0 * n * 8;
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  double apply_ms = 0, spmv_ms = 0;
  int napply = 0;
  auto precond = [&](const double* src, double* dst) {
    k_copy_vec<<<g, 256, 0, s>>>(n, src, dst);
    CKLAUNCH();
    h->prof.launches += 1;
    CK(cudaEventRecord(e0, s));
    apply_any(h, dst, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    apply_ms += ms;
    ++napply;
  };
  // sc: [0] rz, [1] pq, [2] rr, [3] rz_new, [4] bb
  dot(bp, bp, sc + 4);
  const double bnorm = std::sqrt(read(sc + 4));
  int it = 0;
  double rel = 0.0;
  const double tol = h->opts.tol;
  const int maxit = h->opts.maxit;
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(xv, 0, n * sizeof(double), s));
  } else {
    k_copy_vec<<<g, 256, 0, s>>>(n, bp, r);
    CKLAUNCH();
    h->prof.launches += 1;
    precond(r, z);
    k_copy_vec<<<g, 256, 0, s>>>(n, z, p);
    CKLAUNCH();
    int irz = 0, irzn = 3;
    dot(r, z, sc + irz);
    while (it < maxit) {
      CK(cudaEventRecord(e2, s));
      const int pid = h->prof.begin(F_PCG, s);
      k_spmv_dot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, rp, ci, va, p, q, part);
      CKLAUNCH();
      h->prof.launches += 4;
      k_reduce<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, sc + 1);
      CKLAUNCH();
      // alpha = rz / pq
      if (irz != 0) {
        k_copy_vec<<<1, 32, 0, s>>>(1, sc + irz, sc + 0);
        CKLAUNCH();
        h->prof.launches += 1;
        irz = 0;
        irzn = 3;
      }
      k_update_xr<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, sc, xv, r, p, q, part);
      CKLAUNCH();
      k_reduce<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, sc + 2);
      CKLAUNCH();
      h->prof.end(pid, s, 2.0 * h->nnz + 6.0 * n, pcg_bytes, 4);
      CK(cudaEventRecord(e1, s));
      ++it;
      const double rr = read(sc + 2);
      {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e2, e1));
        spmv_ms += ms;
      }
      if (std::sqrt(rr) / bnorm <= tol) {
        k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, rp, ci, va, xv, bp, r);
        CKLAUNCH();
        h->prof.launches += 1;
        dot(r, r, sc + 2);
        if (std::sqrt(read(sc + 2)) / bnorm <= tol) break;
        precond(r, z);
        k_copy_vec<<<g, 256, 0, s>>>(n, z, p);
        CKLAUNCH();
        h->prof.launches += 1;
        dot(r, z, sc + 0);
        continue;
      }
      precond(r, z);
      dot(r, z, sc + irzn);
      k_update_p<<<g, 256, 0, s>>>(n, sc + irzn, sc + irz, z, p);
      CKLAUNCH();
      h->prof.launches += 1;
      std::swap(irz, irzn);
    }
    k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, rp, ci, va, xv, bp, q);
    CKLAUNCH();
    h->prof.launches += 1;
    dot(q, q, sc + 2);
    rel = std::sqrt(read(sc + 2)) / bnorm;
  }
  k_permute<<<g, 256, 0, s>>>(n, perm, xv, io, 0);
  CKLAUNCH();
  h->prof.launches += 1;
  CK(cudaMemcpyAsync(x, io, n * sizeof(double), xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  check_apply(h);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (iters) *iters = it;
  if (relres) *relres = rel;
  h->st.n_cg = it;
  h->st.relres = rel;
  h->st.t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  h->phase_ms[4] = napply ? apply_ms / napply : 0.0;
  h->phase_ms[5] = it ? spmv_ms / it : 0.0;
  if (bnorm != 0.0 && !(rel <= tol)) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%.3e", rel);
    g_err = std::string("PCG stopped at maxit with relative residual ") + buf;
    return SPAND_ERR_NO_CONVERGENCE;
  }
  return SPAND_OK;
  API_END
}

int spand_set_apply_wait(spand_handle h, uint32_t polls, int32_t unreachable) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  h->apply_spin_limit = polls ? polls : kBarrierSpins;
  h->apply_bias = unreachable ? 1u : 0u;
  return SPAND_OK;
}

int spand_set_apply_shape(spand_handle h, int32_t ctas_per_sm) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  if (ctas_per_sm < 0 || ctas_per_sm > kApplyCtasPerSm) {
    g_err = "ctas_per_sm must be in [0, 4]";
    return SPAND_ERR_INVALID_ARG;
  }
  h->apply_ctas = ctas_per_sm;
  if (h->apply_grid > 0 && ctas_per_sm > 0) h->apply_grid = num_sms() * std::min(ctas_per_sm, h->apply_per_sm_max);
  return SPAND_OK;
}

int spand_set_profiling(spand_handle h, int32_t on) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  h->prof.on = on != 0;
  return SPAND_OK;
}

int spand_get_kernel_profile(spand_handle h, int32_t family, double* out4) {
  if (!h || !out4) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  if (family < 0 || family >= F_NFAM) { g_err = "unknown kernel family"; return SPAND_ERR_INVALID_ARG; }
  out4[0] = (double)h->prof.count[family];
  out4[1] = h->prof.ms[family];
  out4[2] = h->prof.flops[family];
  out4[3] = h->prof.bytes[family];
  return SPAND_OK;
}

int spand_reset_kernel_profile(spand_handle h) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  h->prof.reset();
  return SPAND_OK;
}

int spand_get_launch_count(spand_handle h, int64_t* launches) {
  if (!h || !launches) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  *launches = h->prof.launches;
  return SPAND_OK;
}

int spand_sketch_gaussian(uint64_t seed, int32_t step, int32_t cluster, int32_t m, int32_t ell, double* out_dev,
                          void* cuda_stream) {
  API_BEGIN
  g_err.clear();
  if (m < 0 || ell < 0 || step < 0 || cluster < 0)
    throw Fail{SPAND_ERR_INVALID_ARG, "step, cluster, m and ell must be >= 0"};
  if ((int64_t)m * ell == 0) return SPAND_OK;
  if (!out_dev) throw Fail{SPAND_ERR_INVALID_ARG, "out_dev is NULL"};
  if (!is_device_ptr(out_dev)) throw Fail{SPAND_ERR_INVALID_ARG, "out_dev is not device memory"};
  const uint64_t k1 = ((uint64_t)(uint32_t)step << 32) + (uint64_t)(uint32_t)cluster;
  const int64_t blocks = ((int64_t)(m + 3) / 4 * ell + 255) / 256;
  k_sketch_philox<<<(unsigned)std::min<int64_t>(blocks, 8192), 256, 0, (cudaStream_t)cuda_stream>>>(seed, k1, m, ell,
                                                                                                   out_dev);
  CKLAUNCH();
  return SPAND_OK;
  API_END
}

int spand_sampled_outer(spand_handle h, const double* lam_dev, const double* x_dev, double* out_dev,
                        void* cuda_stream) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  API_BEGIN
  g_err.clear();
  const int64_t n = h->n, nnz = h->nnz;
  if (nnz && (!lam_dev || !x_dev || !out_dev)) throw Fail{SPAND_ERR_INVALID_ARG, "null vector"};
  if (nnz == 0) return SPAND_OK;
  if (!h->d_rowptr.p) {  // the original pattern, copied to the device on first use
    h->d_rowptr.ensure((n + 1) * sizeof(int64_t));
    h->d_colind.ensure(nnz * sizeof(int32_t));
    CK(cudaMemcpy(h->d_rowptr.p, h->rowptr.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_colind.p, h->colind.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned g = (unsigned)std::min<int64_t>((n + 7) / 8, 8192);
  k_sampled_outer<<<g, 256, 0, s>>>(n, (const int64_t*)h->d_rowptr.p, (const int32_t*)h->d_colind.p, lam_dev, x_dev,
                                    out_dev);
  CKLAUNCH();
  h->prof.launches += 1;
  CK(cudaStreamSynchronize(s));
  return SPAND_OK;
  API_END
}

int spand_get_tree(spand_handle h, int32_t* perm, int32_t* cluster_ptr, int32_t* cluster_key, int32_t* n_clusters,
                   int32_t* n_steps) {
  if (!h || !n_clusters) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  const Tree& t = h->tree;
  const int nc = (int)t.cluster_ptr.size() - 1;
  *n_clusters = nc;
  if (n_steps) *n_steps = t.L;
  if (perm) std::copy(t.perm.begin(), t.perm.end(), perm);
  if (cluster_ptr) std::copy(t.cluster_ptr.begin(), t.cluster_ptr.end(), cluster_ptr);
  if (cluster_key) std::copy(t.keys.begin(), t.keys.end(), cluster_key);
  return SPAND_OK;
}

int spand_get_step(spand_handle h, int32_t t, int32_t* counts, int32_t* keys, int32_t* child_ptr, int32_t* child_idx,
                   int32_t* elim, int32_t* colour, int32_t* adj_ptr, int32_t* adj_idx, int32_t* adjf_ptr,
                   int32_t* adjf_idx) {
  if (!h || !counts) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  if (t < 1 || t > (int32_t)h->tree.steps.size()) { g_err = "step out of range"; return SPAND_ERR_INVALID_ARG; }
  const StepStruct& s = h->tree.steps[t - 1];
  counts[0] = s.n;
  counts[1] = (int32_t)s.child_idx.size();
  counts[2] = (int32_t)s.adj_idx.size();
  counts[3] = (int32_t)s.adjf_idx.size();
  counts[4] = s.ncolours();
  auto cp = [](const std::vector<int32_t>& v, int32_t* d) { if (d) std::copy(v.begin(), v.end(), d); };
  cp(s.keys, keys);
  cp(s.child_ptr, child_ptr);
  cp(s.child_idx, child_idx);
  cp(s.elim, elim);
  cp(s.colour, colour);
  cp(s.adj_ptr, adj_ptr);
  cp(s.adj_idx, adj_idx);
  cp(s.adjf_ptr, adjf_ptr);
  cp(s.adjf_idx, adjf_idx);
  return SPAND_OK;
}

int spand_get_ranks(spand_handle h, int32_t t, int32_t* sizes_before, int32_t* sizes_after) {
  if (!h) { g_err = "null handle"; return SPAND_ERR_INVALID_ARG; }
  if (!h->factored) { g_err = "not factorized"; return SPAND_ERR_STATE; }
  if (t < 1 || t > (int32_t)h->sizes_before.size()) { g_err = "step out of range"; return SPAND_ERR_INVALID_ARG; }
  if (sizes_before) std::copy(h->sizes_before[t - 1].begin(), h->sizes_before[t - 1].end(), sizes_before);
  if (sizes_after) std::copy(h->sizes_after[t - 1].begin(), h->sizes_after[t - 1].end(), sizes_after);
  return SPAND_OK;
}

int spand_get_stats(spand_handle h, spand_stats* st) {
  if (!h || !st) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  h->st.apply_ctas_per_sm = h->apply_ctas;
  *st = h->st;
  return SPAND_OK;
}

int spand_get_phase_times(spand_handle h, double* out6) {
  if (!h || !out6) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  for (int i = 0; i < 6; ++i) out6[i] = h->phase_ms[i];
  return SPAND_OK;
}

void spand_destroy(spand_handle h) { delete h; }

int spand_analyze_batch(int32_t k, const spand_problem* probs, const spand_opts* opts, spand_handle* out) {
  g_err.clear();
  if (k < 0) { g_err = "k must be >= 0"; return SPAND_ERR_INVALID_ARG; }
  if (k == 0) return SPAND_OK;
  if (!probs || !opts || !out) { g_err = "null argument"; return SPAND_ERR_INVALID_ARG; }
  for (int32_t i = 0; i < k; ++i) out[i] = nullptr;
  std::vector<int> rc(k, SPAND_OK);
  std::vector<std::string> msg(k);
  const int nth = (int)std::max(1u, std::min<unsigned>((unsigned)k, std::thread::hardware_concurrency()));
  auto work = [&](int w) {  // problems w, w + nth, ... (analysis is host-only and handle-local)
    for (int32_t i = w; i < k; i += nth) {
      const spand_problem& p = probs[i];
      rc[i] = spand_analyze(p.n, p.rowptr, p.colind, p.vals, p.coords, p.dim, &opts[i], &out[i]);
      if (rc[i] != SPAND_OK) msg[i] = spand_last_error();
    }
  };
  try {
    std::vector<std::thread> pool;
    for (int w = 1; w < nth; ++w) pool.emplace_back(work, w);
    work(0);
    for (auto& t : pool) t.join();
  } catch (const std::exception& e) {  // thread creation failed
    for (int32_t i = 0; i < k; ++i) {
      delete out[i];
      out[i] = nullptr;
    }
    g_err = std::string("analyze_batch: ") + e.what();
    return SPAND_ERR_OOM;
  }
  for (int32_t i = 0; i < k; ++i)
    if (rc[i] != SPAND_OK) {
      const int code = rc[i];
      g_err = "problem " + std::to_string(i) + ": " + msg[i];
      for (int32_t j = 0; j < k; ++j) {
        delete out[j];
        out[j] = nullptr;
      }
      return code;
    }
  return SPAND_OK;
}

}  // extern "C"
