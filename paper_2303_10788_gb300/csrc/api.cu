#include <thread>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <functional>
#include <exception>
#include <mutex>
// C ABI of the circuit-cutting hot path (declared in include/ccs.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "abi_guard.hpp"
#include "kernels.cuh"
#include "plan.hpp"

using namespace ccs;

struct ccs_ctx_s {
  int device = 0;
  bool host_only = false;   // device < 0: planning only, no GPU work
  cudaStream_t stream = nullptr;
  ccs_allocator alloc{nullptr, nullptr, nullptr};
  bool own_alloc = true;
  int sm_count = 0;
  size_t smem_optin = 0;
  std::string err;
  ccs_mpnn cut_model = nullptr;   // learned cut scorer (not owned)
  // autotuner results: shape bucket -> (Clifford threads per CTA, shots per sampler CTA)
  std::map<std::tuple<int, int, unsigned, int>, std::tuple<int, int, int, int, int>> tuned;
  // second stream for the statevector branch (forked from / joined into `stream`)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // stage timing (CUDA events around each launch on the context stream)
  bool profiling = false;
  cudaEvent_t ev[16] = {};
  int n_ev = 0;
  float stage_ms[8] = {};
  int stage_mask = 0;   // stages recorded by the last profiled call
  // pinned staging buffer for plan uploads (one host->device copy per batch);
  // the event marks the end of the last copy out of it
  char* pinned = nullptr;
  size_t pinned_bytes = 0;
  cudaEvent_t upload_ev = nullptr;
  bool upload_pending = false;
};

cudaStream_t ccs::c_stream(ccs_ctx c) { return c->stream; }

namespace {
enum Stage { ST_CLIFFORD = 0, ST_SAMPLE = 1, ST_STATEVEC = 2, ST_FOLD = 3, ST_RECOMB = 4, ST_OPERANDS = 5, ST_N = 6 };
void stage_begin(ccs_ctx c, int st) {
  if (!c->profiling) return;
  if (!c->ev[2 * st]) { cudaEventCreate(&c->ev[2 * st]); cudaEventCreate(&c->ev[2 * st + 1]); }
  cudaEventRecord(c->ev[2 * st], c->stream);
}
void stage_end(ccs_ctx c, int st) {
  if (!c->profiling) return;
  cudaEventRecord(c->ev[2 * st + 1], c->stream);
  c->stage_mask |= 1 << st;
}
}  // namespace

namespace {

int fail(ccs_ctx c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(ccs_ctx c, cudaError_t e, const char* where) {
  return fail(c, CCS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device memory of contexts created without an allocator: one stream-ordered
// pool per device shared by them, which keeps freed memory for reuse
// (release threshold unlimited) instead of handing it back to the driver at
// every synchronisation as the device's default pool does, so that plans and
// results made every step reuse their memory.  ccs_destroy trims it.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaMemPool_t lib_pool(int device) {
  if (device < 0 || device >= kMaxPoolDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[device]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[device] = pool;
  }
  return g_pools[device];
}

void* dalloc(ccs_ctx c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (!c->own_alloc) return c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
  void* p = nullptr;
  cudaMemPool_t pool = lib_pool(c->device);
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, c->stream) : cudaMallocAsync(&p, bytes, c->stream);
  return e == cudaSuccess ? p : nullptr;
}

void dfree(ccs_ctx c, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (!c->own_alloc) c->alloc.free(p, bytes, (void*)c->stream, c->alloc.user);
  else cudaFreeAsync(p, c->stream);
}

// Device memory of one plan or result.  Small requests are carved, 256-byte
// aligned, out of 1 MiB blocks so a plan or result costs a handful of
// allocator calls; large ones get their own block.
struct Allocs {
  static constexpr size_t kBlock = 1 << 20, kSmall = 128 << 10;
  ccs_ctx ctx = nullptr;
  std::vector<std::pair<void*, size_t>> list;
  char* cur = nullptr;
  size_t left = 0;
  template <class T>
  T* get(size_t count) {
    const size_t bytes = (std::max<size_t>(count * sizeof(T), 1) + 255) & ~(size_t)255;
    if (bytes > kSmall) {
      void* p = dalloc(ctx, bytes);
      if (p) list.push_back({p, bytes});
      return (T*)p;
    }
    if (bytes > left) {
      void* p = dalloc(ctx, kBlock);
      if (!p) return nullptr;
      list.push_back({p, kBlock});
      cur = (char*)p;
      left = kBlock;
    }
    T* p = (T*)cur;
    cur += bytes;
    left -= bytes;
    return p;
  }
  void release() {
    for (auto& a : list) dfree(ctx, a.first, a.second);
    list.clear();
    cur = nullptr;
    left = 0;
  }
};

// Host worker pool: threads created once (up to hardware_concurrency, at most
// 32) and kept for the life of the process, so a plan build spawns no thread
// and each worker keeps its scratch buffers warm.  Several callers may post
// jobs at once; a caller works on its own job too, so a job finishes even
// when every worker is busy (and a job posted from inside a job cannot wait
// on itself).  A job lives on its caller's stack: the caller returns only
// when every item is done and no worker still holds the job (both counted
// under the pool's mutex, under which workers also pick jobs up).
class HostPool {
 public:
  struct Job {
    const std::function<void(int)>* f = nullptr;
    int n = 0;
    int holders = 0;                 // workers inside work() (guarded by the pool's mutex)
    std::atomic<int> next{0}, done{0};
    std::exception_ptr first;
    std::mutex err_mu;
    void work() {
      for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) {
        try {
          (*f)(i);
        } catch (...) {
          std::lock_guard<std::mutex> lk(err_mu);
          if (!first) first = std::current_exception();
        }
        done.fetch_add(1);
      }
    }
  };
  static HostPool& get() {
    static HostPool* pool = new HostPool();   // never destroyed: detached workers outlive static destructors
    return *pool;
  }
  int size() const { return (int)workers_.size(); }
  void run(Job& j) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      jobs_.push_back(&j);
    }
    work_cv_.notify_all();
    j.work();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return j.done.load() == j.n && j.holders == 0; });
    for (auto it = jobs_.begin(); it != jobs_.end(); ++it)
      if (*it == &j) { jobs_.erase(it); break; }
  }

 private:
  HostPool() {
    const unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    for (unsigned t = 1; t < hw; ++t) workers_.emplace_back([this] { loop(); });
    for (auto& w : workers_) w.detach();
  }
  void loop() {
    for (;;) {
      Job* j = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        work_cv_.wait(lk, [&] {
          for (Job* x : jobs_)
            if (x->next.load() < x->n) { j = x; return true; }
          return false;
        });
        ++j->holders;
      }
      j->work();
      {
        std::lock_guard<std::mutex> lk(mu_);
        --j->holders;                // the worker's last access to the job
      }
      done_cv_.notify_all();
    }
  }
  std::mutex mu_;
  std::condition_variable work_cv_, done_cv_;
  std::deque<Job*> jobs_;
  std::vector<std::thread> workers_;
};

// f(0..n-1) on the host pool (inline for n = 1); an exception in any item is
// carried to the calling thread (the first one wins; the other items still run).
template <class F>
void parallel_for(int n, F&& f) {
  if (n <= 1) {
    if (n == 1) f(0);
    return;
  }
  HostPool& pool = HostPool::get();
  if (pool.size() == 0) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  const std::function<void(int)> fn = [&](int i) { f(i); };
  HostPool::Job j;
  j.f = &fn;
  j.n = n;
  pool.run(j);
  if (j.first) std::rethrow_exception(j.first);
}

// Host arrays gathered into one pinned buffer and sent with one copy.
struct Staging {
  struct Item { const void* src; size_t bytes, off; void** out; };
  std::vector<Item> items;
  size_t total = 0;
  template <class T>
  void add(const std::vector<T>& h, T** out) {
    const size_t bytes = h.size() * sizeof(T);
    items.push_back({h.data(), bytes, total, reinterpret_cast<void**>(out)});
    total += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
  }
  bool commit(ccs_ctx c, Allocs& A) {
    if (items.empty()) return true;
    char* d = A.get<char>(total);
    if (!d) return false;
    // the previous copy out of the staging buffer must be done before reuse
    // (waits for that copy only, not for other work on the stream)
    if (!upload_wait(c)) return false;
    if (c->pinned_bytes < total) {
      if (c->pinned) cudaFreeHost(c->pinned);
      c->pinned = nullptr;
      c->pinned_bytes = 0;
      if (cudaMallocHost(&c->pinned, total) != cudaSuccess) return false;
      c->pinned_bytes = total;
    }
    for (auto& it : items) {
      if (it.bytes) std::memcpy(c->pinned + it.off, it.src, it.bytes);
      *it.out = d + it.off;
    }
    if (cudaMemcpyAsync(d, c->pinned, total, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) return false;
    if (!c->upload_ev && cudaEventCreateWithFlags(&c->upload_ev, cudaEventDisableTiming) != cudaSuccess) return false;
    if (cudaEventRecord(c->upload_ev, c->stream) != cudaSuccess) return false;
    c->upload_pending = true;
    return true;
  }
  static bool upload_wait(ccs_ctx c) {
    if (!c->upload_pending) return true;
    if (cudaEventSynchronize(c->upload_ev) != cudaSuccess) return false;
    c->upload_pending = false;
    return true;
  }
};

template <class T>
bool upload(ccs_ctx c, Allocs& A, const std::vector<T>& h, T** out) {
  *out = A.get<T>(std::max<size_t>(h.size(), 1));
  if (!*out) return false;
  if (!h.empty() &&
      cudaMemcpyAsync(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return false;
  return true;
}

}  // namespace

struct ccs_plan_s {
  ccs_ctx ctx = nullptr;
  bool host_only = false;
  std::vector<Problem> problems;
  std::vector<Frag> frags;
  std::vector<FragDev> fdev;
  std::vector<ProblemDev> pdev;
  DevPlan dp{};
  Allocs A;
  long long n_spaces = 0, n_counts = 0, n_dist = 0, n_zval = 0, n_tab = 0, n_T = 0, n_body = 0;
  long long n_zimg = 0;             // uint64 words of Z images
  long long n_pbasis = 0;           // uint32 words of projected shared-row bases
  long long n_marg = 0, n_zexp = 0;
  std::vector<long long> t_prefix, out_prefix, z_prefix, r_prefix, blk_prefix;
  std::vector<int2> direct_items;   // (problem, hub-output slice) contracted leaf by leaf
  int2* d_direct_items = nullptr;
  long long direct_stage_floats = 0;
  int chain = 0;                    // some problem takes the R / GEMM / reduce chain
  long long* d_r_prefix = nullptr;
  long long* d_blk_prefix = nullptr;
  long long r_total = 0, part_total = 0, gemm_blocks = 0, rt_total = 0;
  std::vector<long long> s_prefix;
  long long* d_s_prefix = nullptr;
  int max_tile_smem = 0;
  long long* d_t_prefix = nullptr;
  long long* d_out_prefix = nullptr;
  long long* d_z_prefix = nullptr;
  int cliff_smem_words = 0, max_nc_n = 1;
  int nc_basis_chunk = 1;           // basis combinations per statevector item
  int body_smem_words = 0;          // variant kernel started from a shared body (no op staging)
  FoldSet fold_cliff{}, fold_nc{}, fold_hubs{}, fold_hubs_nc{}, fold_others{};
  int2* d_items_hub = nullptr;      // Clifford hub variants (fused sampler)
  int2* d_items_plain = nullptr;    // other Clifford variants (sampler -> counts)
  int n_items_hub = 0, n_items_plain = 0, max_hub_nA = 0;
  bool hub_bytes_ok = true;         // every hub fits the byte-counter sampler
  long long n_counts_plain = 0;     // counts of non-hub Clifford fragments come first
  long long n_dist_nc = 0;          // distributions of statevector fragments come first
  long long n_dist_stitch = 0;      // ... then non-hub Clifford fragments (all a stitched evaluation needs)
  long long n_qrows = 0;            // operand-row flags of the Clifford hubs
  bool stitch_ok = true;            // every Clifford hub has at most 4 quantum outputs
  bool tableau_fits = true;         // every Clifford fragment's whole tableau fits in shared memory
  bool all_star = true;
  ~ccs_plan_s() { A.release(); }
};

struct ccs_res_s {
  ccs_plan plan = nullptr;
  DevRes dr{};
  EvalParams ep{};
  bool have_tabs = false;
  bool have_counts = false;
  bool counts_full = false;   // counts include the hubs' (kept for inspection)
  long long dist_len = 0;     // floats of the distribution buffer (statevector fragments first,
                              // then non-hub Clifford, then hub Clifford fragments)
  Allocs A;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;   // kernel nodes of the captured graph
  cudaGraphExec_t rgraph = nullptr;   // recombination graph
  int rgraph_key = -1;
  long long rgraph_launches = 0;
  EvalParams graph_key{};
  int graph_valid = 0;
  int cliff_threads = 256;
  int cliff_words = 1;        // words per op per thread in the tableau kernel
  int sample_spc = 4096;
  int hub_threads = 512;      // threads of the fused hub sampler CTA (either counter width)
  bool hub_bytes = false;     // use the byte-counter hub sampler (64 KB of counters at |A| = 16)
  bool variant_path = false;  // autotuned: every variant simulates its whole circuit (small plans)
  float* scratch = nullptr;   // recombination: R operand + split-K partials
  uint16_t* rt_scratch = nullptr;   // bf16 R'^T of tensor-core-eligible problems
  int eval_i16 = 0;           // hub_i16 of the last evaluation (the one its graph holds)
  int ml_applied = 0;         // 1 + the fragment selection of ccs_ml_correct since the evaluation
  struct MlCache {            // device records of the last ccs_ml_correct selection
    int key = -1;
    MlFrag* d_frags = nullptr;
    int n_frags = 0;
    std::vector<MlGroup> groups;
    float* scratch = nullptr;
    size_t scratch_len = 0;
    double* theta = nullptr;
    FoldSet leaves{nullptr, nullptr, 0, 0};   // corrected star leaves: T' is formed again
    bool i16_hub = false;
  } ml;
  ~ccs_res_s() {
    if (graph) cudaGraphExecDestroy(graph);
    if (rgraph) cudaGraphExecDestroy(rgraph);
    A.release();
  }
};

// Score up to 16 candidate cut sets with the learned model; index of the
// smallest predicted time.
namespace ccs {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ccs

// The learned choice among the greedy candidates the greedy estimate allows
// (at most 16x the cheapest estimate, at most 16 of them): featurize each,
// one scorer forward on the GPU, take the smallest predicted log time.
static int learned_pick(ccs_ctx c, const Problem& P, const std::vector<CutCandidate>& cands, int* pick) {
  std::vector<int> idx;
  for (int i = 0; i < (int)cands.size() && (int)idx.size() < 16; ++i)
    if (cands[i].cost <= 16.0 * cands.front().cost) idx.push_back(i);
  *pick = 0;
  if (idx.size() < 2) return CCS_OK;
  const int nc = (int)idx.size();
  // the interaction graph once, the candidates' node features on host threads
  const GraphBase g = graph_base(P);
  std::vector<std::vector<float>> xs(nc), gs(nc);
  std::vector<int> rcs(nc, CCS_OK);
  std::vector<std::string> errs(nc);
  parallel_for(nc, [&](int i) { rcs[i] = featurize_nodes(P, g, cands[idx[i]].cuts, xs[i], gs[i], errs[i]); });
  for (int i = 0; i < nc; ++i)
    if (rcs[i] != CCS_OK) return fail(c, rcs[i], errs[i]);
  std::vector<float> X, val, valt, glob;
  std::vector<int> rowptr{0}, col, goff{0};
  for (int i = 0; i < nc; ++i) {
    const int base = goff.back(), e0 = rowptr.back();
    X.insert(X.end(), xs[i].begin(), xs[i].end());
    for (size_t r = 1; r < g.rowptr.size(); ++r) rowptr.push_back(e0 + g.rowptr[r]);
    for (int cc : g.col) col.push_back(base + cc);
    val.insert(val.end(), g.val.begin(), g.val.end());
    valt.insert(valt.end(), g.val_t.begin(), g.val_t.end());
    glob.insert(glob.end(), gs[i].begin(), gs[i].end());
    goff.push_back(base + (int)P.n_qubits);
  }
  ccs_graph_batch b{goff.back(), nc, X.data(), rowptr.data(), col.data(), val.data(), valt.data(), goff.data(),
                    glob.data()};
  std::vector<float> pred(nc);
  if (mpnn_predict(c->cut_model, &b, pred.data()) != CCS_OK) return fail(c, CCS_ERR_CUDA, "cut model forward");
  *pick = idx[std::min_element(pred.begin(), pred.end()) - pred.begin()];
  return CCS_OK;
}

extern "C" {

int ccs_set_cut_model(ccs_ctx c, ccs_mpnn net) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c) return CCS_ERR_INVALID_ARG;
    c->cut_model = net;
    return CCS_OK;
  });
}

int ccs_featurize(ccs_ctx c, const ccs_problem* q, const ccs_cut* cuts, int n_cuts, float* x, int32_t* rowptr,
                  int32_t* col, float* val, float* val_t, int cap_nnz, float* glob) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !q || (n_cuts > 0 && !cuts) || !x || !rowptr || !glob) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    Problem P;
    P.n_qubits = q->n_qubits;
    std::string err;
    int rc = check_circuit(*q, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    rc = load_gates(q->gates, q->n_gates, P.gates, P.gparam, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    P.marginal.assign(q->marginal, q->marginal + q->n_marginal);
    std::vector<ccs_cut> cs(cuts, cuts + std::max(0, n_cuts));
    std::vector<float> X, v, vt, g;
    std::vector<int> rp, cl;
    rc = featurize(P, cs, X, rp, cl, v, vt, g, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    if ((int)cl.size() > cap_nnz) return fail(c, CCS_ERR_INVALID_ARG, "edge buffer too small");
    std::copy(X.begin(), X.end(), x);
    std::copy(rp.begin(), rp.end(), rowptr);
    std::copy(cl.begin(), cl.end(), col);
    if (val) std::copy(v.begin(), v.end(), val);
    if (val_t) std::copy(vt.begin(), vt.end(), val_t);
    std::copy(g.begin(), g.end(), glob);
    return (int)cl.size();
  });
}

long long ccs_launch_count(void) { return launch_count(); }

const char* ccs_version(void) { return "ccs 0.1 (sm_103a)"; }

int ccs_create(ccs_ctx* out, int device, void* cuda_stream, const ccs_allocator* alloc) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!out) return CCS_ERR_INVALID_ARG;
    *out = nullptr;
    if (device < 0) {   // host-only context: fragments and plans can be built and inspected
      ccs_ctx c = new ccs_ctx_s();
      c->device = -1;
      c->host_only = true;
      c->smem_optin = 227 * 1024;
      *out = c;
      return CCS_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CCS_ERR_CUDA;
    ccs_ctx c = new ccs_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (alloc && alloc->alloc && alloc->free) {
      c->alloc = *alloc;
      c->own_alloc = false;
    }
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return CCS_ERR_CUDA; }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
      delete c;
      return CCS_ERR_CUDA;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    *out = c;
    return CCS_OK;
  });
}

void ccs_destroy(ccs_ctx c) {
  if (!c) return;
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->upload_ev) cudaEventDestroy(c->upload_ev);
  if (c->own_alloc && !c->host_only && c->device >= 0 && c->device < kMaxPoolDevices) {
    std::lock_guard<std::mutex> lk(g_pool_mu);   // hand the pool's unused memory back
    if (g_pools[c->device]) cudaMemPoolTrimTo(g_pools[c->device], 0);
  }
  delete c;
}

int ccs_set_profiling(ccs_ctx c, int on) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c) return CCS_ERR_INVALID_ARG;
    if (c->host_only) return fail(c, CCS_ERR_UNSUPPORTED, "host-only context");
    c->profiling = on != 0;
    c->stage_mask = 0;
    return CCS_OK;
  });
}

int ccs_get_stage_times(ccs_ctx c, double* ms, int cap) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !ms || cap < ST_N) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (c->host_only || !c->profiling) return fail(c, CCS_ERR_UNSUPPORTED, "profiling is off");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    for (int st = 0; st < ST_N; ++st) {
      ms[st] = -1.0;
      if (c->stage_mask & (1 << st)) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev[2 * st], c->ev[2 * st + 1]) == cudaSuccess) ms[st] = t;
      }
    }
    return ST_N;
  });
}

const char* ccs_last_error(ccs_ctx c) { return c ? c->err.c_str() : "null context"; }

int ccs_build_fragments(ccs_ctx c, const ccs_problem* probs, int n_problems, const ccs_cut_opts* opts,
                        ccs_plan* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !out || (n_problems > 0 && !probs) || n_problems < 0) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    *out = nullptr;
    if (!c->host_only) cudaSetDevice(c->device);
    ccs_cut_opts o{kMaxCuts, 10, 0};
    if (opts) o = *opts;
    // the plan is freed on every early return and on an exception
    std::unique_ptr<ccs_plan_s> owned(new ccs_plan_s());
    ccs_plan plan = owned.get();
    plan->ctx = c;
    plan->A.ctx = c;
    std::string err;
    // Per problem, on host threads: parse, cut search (if asked), fragment
    // and compile.  Results are joined in problem order, so the plan does not
    // depend on the thread count.
    const int np = n_problems;
    std::vector<Problem> pr(np);
    std::vector<std::vector<Frag>> pf(np);
    std::vector<std::vector<CutCandidate>> pc(np);
    std::vector<int> prc(np, CCS_OK);
    std::vector<std::string> perr(np);
    parallel_for(np, [&](int pi) {
      const ccs_problem& q = probs[pi];
      Problem& P = pr[pi];
      P.n_qubits = q.n_qubits;
      prc[pi] = check_circuit(q, perr[pi]);
      if (prc[pi] != CCS_OK) return;
      prc[pi] = load_gates(q.gates, q.n_gates, P.gates, P.gparam, perr[pi]);
      if (prc[pi] != CCS_OK) return;
      P.marginal.assign(q.marginal, q.marginal + q.n_marginal);
      for (uint32_t z = 0; z < q.n_zstrings; ++z)
        P.zstrings.emplace_back(q.zstring_qubits + q.zstring_offsets[z], q.zstring_qubits + q.zstring_offsets[z + 1]);
      if (q.n_cuts >= 0) {
        if (q.n_cuts > 0 && !q.cuts) { prc[pi] = CCS_ERR_INVALID_ARG; perr[pi] = "null cut list"; return; }
        P.cuts.assign(q.cuts, q.cuts + q.n_cuts);
        if ((int)P.cuts.size() > o.max_cuts) { prc[pi] = CCS_ERR_TOO_MANY_CUTS; perr[pi] = "too many cuts"; return; }
      } else {
        CutSearchOpts so;
        so.max_cuts = std::min(o.max_cuts, kMaxCuts);
        so.max_nc_width = std::min(o.max_nc_width > 0 ? o.max_nc_width : 10, kMaxNCWidth);
        prc[pi] = greedy_cuts(P, so, pc[pi], perr[pi]);
        if (prc[pi] != CCS_OK) return;
        P.cuts = pc[pi].front().cuts;
      }
    });
    for (int pi = 0; pi < np; ++pi)
      if (prc[pi] != CCS_OK) { return fail(c, prc[pi], perr[pi]); }
    // the learned choice runs the scorer on the GPU: one problem at a time
    if (o.use_learned && c->cut_model && !c->host_only)
      for (int pi = 0; pi < np; ++pi)
        if (pc[pi].size() > 1) {
          int pick = 0;
          int rc = learned_pick(c, pr[pi], pc[pi], &pick);
          if (rc != CCS_OK) { return rc; }
          pr[pi].cuts = pc[pi][pick].cuts;
        }
    parallel_for(np, [&](int pi) {
      prc[pi] = fragment_problem(pr[pi], pi, pf[pi], perr[pi]);
      if (prc[pi] != CCS_OK) return;
      for (auto& f : pf[pi]) {
        if (f.clifford) compile_clifford(f);
        else compile_nc(f);
      }
    });
    for (int pi = 0; pi < np; ++pi)
      if (prc[pi] != CCS_OK) { return fail(c, prc[pi], "problem " + std::to_string(pi) + ": " + perr[pi]); }
    for (int pi = 0; pi < np; ++pi) {
      const int base = (int)plan->frags.size();      // fragment ids become plan-global
      for (auto& id : pr[pi].frag_ids) id += base;
      for (auto& f : pf[pi]) plan->frags.push_back(std::move(f));
      plan->problems.push_back(std::move(pr[pi]));
    }

    // --- flatten ---------------------------------------------------------------
    std::vector<CliffordOp> cops;
    std::vector<NCOp> nops;
    std::vector<int> moments, wires, zoffs;
    std::vector<int2> items_c, items_nc, items_b, items_z, items_p, zblocks;
    std::vector<int> nc_frags;
    std::vector<int> cliff_frags;
    int img_words_max = 0, body_words_max = 0;
    int max_body_stage = 0, max_moment_ops = 1;
    int max_body_cols = 0;
    std::vector<long long> cost_c, cost_nc;
    {   // sizes first: every array below is filled without reallocation
      size_t n_cops = 0, n_nops = 0, n_mom = 0, n_var = 0, n_wire = 0;
      for (const Frag& f : plan->frags) {
        n_cops += f.cops.size();
        n_nops += f.nops.size();
        n_mom += f.moment_start.size();
        n_wire += 2 * f.qout_wire.size() + f.marg_wire.size() + f.qin_wire.size();
        for (auto& zw : f.zwires) n_wire += zw.size();
        if (f.clifford) n_var += f.n_variants();
      }
      cops.reserve(n_cops);
      nops.reserve(n_nops);
      moments.reserve(n_mom);
      wires.reserve(n_wire);
      items_c.reserve(n_var);
      cost_c.reserve(n_var);
      plan->fdev.reserve(plan->frags.size());
    }
    for (size_t fi = 0; fi < plan->frags.size(); ++fi) {
      Frag& f = plan->frags[fi];
      FragDev d{};
      d.n = f.n();
      d.Wh = (d.n + 63) / 64;
      d.W = 2 * d.Wh;
      d.nA = f.n_meas();
      d.m = (int)f.marg_wire.size();
      d.qin = (int)f.qin_wire.size();
      d.qout = (int)f.qout_wire.size();
      d.nv = f.n_variants();
      d.clifford = f.clifford ? 1 : 0;
      d.problem = f.problem;
      d.findex = f.index;
      d.ops_off = f.clifford ? (int)cops.size() : (int)nops.size();
      d.mom_off = (int)moments.size();
      d.n_moments = f.n_moments();
      for (int x : f.moment_start) moments.push_back(x);
      if (f.clifford) cops.insert(cops.end(), f.cops.begin(), f.cops.end());
      else nops.insert(nops.end(), f.nops.begin(), f.nops.end());
      d.A_off = (int)wires.size();
      for (int w : f.marg_wire) wires.push_back(w);
      for (int w : f.qout_wire) wires.push_back(w);
      d.qin_off = (int)wires.size();
      for (int w : f.qin_wire) wires.push_back(w);
      d.qout_off = (int)wires.size();
      for (int w : f.qout_wire) wires.push_back(w);
      d.nz = (int)f.zwires.size();
      d.zw_off = (int)zoffs.size();
      for (auto& zw : f.zwires) {
        zoffs.push_back((int)wires.size());
        for (int w : zw) wires.push_back(w);
      }
      zoffs.push_back((int)wires.size());
      d.n_slots = (int)f.slots.size();
      for (int j = 0; j < d.n_slots; ++j) {
        d.slot_code[j] = (f.slot_kind[j] << 8) | f.slot_idx[j];
        d.slot_cut[j] = f.slots[j];
      }
      for (int j = 0; j < d.m; ++j) d.marg_pos[j] = f.marg_pos[j];
      const long long outs = 1ll << d.nA;
      if (f.clifford) {
        d.space_off = plan->n_spaces;
        plan->n_spaces += d.nv;
        d.counts_off = plan->n_counts;
        plan->n_counts += (long long)d.nv * outs;
        d.tab_off = plan->n_tab;
        plan->n_tab += (long long)d.nv * (2 * d.n + 3) * d.W;
        d.body_off = plan->n_body;      // even: (2n+3)*W is even, so 16-byte aligned
        plan->n_body += (long long)(2 * d.n + 3) * d.W;
        d.rb_off = (long long)kRowBasisWords * (long long)cliff_frags.size();
        cliff_frags.push_back((int)fi);
        d.pb_off = -1;
        if (d.qout <= kMaxPbQout) {
          int combos = 1;
          for (int o = 0; o < d.qout; ++o) combos *= 3;
          d.pb_off = plan->n_pbasis;
          plan->n_pbasis += 25ll * combos;
          for (int pc = 0; pc < combos; ++pc) items_p.push_back(make_int2((int)fi, pc));
        }
        {   // Z images: every string, X, Y, Z of every quantum output, Z of every marginal wire
          const int ni = d.nz + 3 * d.qout + d.m;
          d.zimg_off = plan->n_zimg;
          plan->n_zimg += (long long)ni * (2 * d.Wh + 1);
          img_words_max = std::max(img_words_max, ni * (2 * d.Wh + 1));
          body_words_max = std::max(body_words_max, (2 * d.n + 3) * d.W);
          for (int k = 0; k < ni; ++k) items_z.push_back(make_int2((int)fi, k));
          if (d.nz > 0)
            for (int v = 0; v < d.nv; v += zblock_variants(d.nz)) zblocks.push_back(make_int2((int)fi, v));
        }
        max_body_stage = std::max(max_body_stage, 2 * d.n + 3 + (int)f.cops.size() + (d.n_moments + 2) / 2 + 1);
        for (int mm = 0; mm < f.n_moments(); ++mm)
          max_moment_ops = std::max(max_moment_ops, f.moment_start[mm + 1] - f.moment_start[mm]);
        for (int w = 0; w < d.W; ++w) items_b.push_back(make_int2((int)fi, w));
        max_body_cols = std::max(max_body_cols, 2 * d.n + 3);
        const int words = (2 * d.n + 3) * d.W + (d.n + 1) / 2 + 2;
        const int staged = words + (int)f.cops.size() + (d.n_moments + 2) / 2 + 2;   // + op stream
        plan->cliff_smem_words =
            std::max(plan->cliff_smem_words, (size_t)staged * 8 <= c->smem_optin ? staged : words);
        plan->body_smem_words = std::max(plan->body_smem_words, words);
        for (int v = 0; v < d.nv; ++v) {
          items_c.push_back(make_int2((int)fi, v));
          cost_c.push_back((long long)d.W * (d.n_moments + 4) * std::max(1, d.n / 16) + d.nz * 4 + d.nA * d.n);
        }
      } else {
        d.space_off = d.counts_off = d.tab_off = d.body_off = d.rb_off = d.zimg_off = d.pb_off = -1;
        plan->max_nc_n = std::max(plan->max_nc_n, d.n);
        nc_frags.push_back((int)fi);
      }
      d.dist_off = plan->n_dist;
      plan->n_dist += (long long)d.nv * outs;
      d.zval_off = plan->n_zval;
      plan->n_zval += (long long)d.nv * d.nz * (1ll << d.qout);
      d.T_off = (plan->n_T + 63) & ~63ll;     // 256-byte aligned (TMA needs 16)
      plan->n_T = d.T_off + (1ll << d.m) * (1ll << (2 * d.n_slots));
      plan->fdev.push_back(d);
    }
    {   // distributions: statevector fragments first (all a sampled evaluation needs), then Clifford
      long long off = 0;
      for (auto& f : plan->fdev)
        if (!f.clifford) { f.dist_off = off; off += (long long)f.nv << f.nA; }
      plan->n_dist_nc = off;
    }
    // a per-variant tableau (kept tableaus, per-variant bodies) must fit in
    // shared memory; the shared-body path has no such limit (checked at evaluation)
    plan->tableau_fits = (size_t)plan->cliff_smem_words * 8 <= c->smem_optin || items_c.empty();
    // Items costliest first, ties in insertion order.  A fragment's items are
    // consecutive and cost the same, so the runs of equal cost are sorted
    // stably instead of the items (the same order, far fewer comparisons).
    auto sort_items = [](std::vector<int2>& it, std::vector<long long>& cost) {
      std::vector<std::pair<size_t, size_t>> runs;
      for (size_t i = 0; i < it.size();) {
        size_t j = i + 1;
        while (j < it.size() && cost[j] == cost[i]) ++j;
        runs.push_back({i, j});
        i = j;
      }
      std::stable_sort(runs.begin(), runs.end(),
                       [&](const std::pair<size_t, size_t>& a, const std::pair<size_t, size_t>& b) {
                         return cost[a.first] > cost[b.first];
                       });
      std::vector<int2> out;
      out.reserve(it.size());
      for (auto& r : runs) out.insert(out.end(), it.begin() + r.first, it.begin() + r.second);
      it.swap(out);
    };
    sort_items(items_c, cost_c);
    // Non-Clifford items: with enough variants to fill the GPU, one item per
    // preparation combination (the gates run once, every basis combination of
    // the outputs is applied to a copy of the state); otherwise one per variant
    // (latency: no serial basis tails).
    {
      long long nc_total = 0;
      for (int fi : nc_frags) nc_total += plan->fdev[fi].nv;
      const int chunk = nc_total > 2ll * std::max(c->sm_count, 148) ? 1 << 30 : 1;
      plan->nc_basis_chunk = chunk;
      for (int fi : nc_frags) {
        const FragDev& d = plan->fdev[fi];
        const int n_prep = 1 << (2 * d.qin), n_basis = d.nv / n_prep;
        const long long nops = plan->frags[fi].nops.size();
        for (int b0 = 0; b0 < n_basis; b0 += std::min(chunk, n_basis))
          for (int pc = 0; pc < n_prep; ++pc) {
            items_nc.push_back(make_int2(fi, pc + n_prep * b0));
            cost_nc.push_back((1ll << d.n) * (nops + 4 + 8ll * std::min(chunk, n_basis - b0)));
          }
      }
    }
    sort_items(items_nc, cost_nc);

    int f0 = 0;
    plan->t_prefix.push_back(0);
    plan->out_prefix.push_back(0);
    plan->z_prefix.push_back(0);
    plan->r_prefix.push_back(0);
    plan->blk_prefix.push_back(0);
    for (auto& f : plan->fdev) {
      plan->t_prefix.push_back(plan->t_prefix.back() + (1ll << f.m) * (1ll << (2 * f.n_slots)));
    }
    // roles in star problems: the hub's contraction operand is Q, the others' T'
    {
      int f0r = 0;
      for (auto& P : plan->problems) {
        const int nfr = (int)P.frag_ids.size();
        if (P.hub >= 0)
          for (int l = 0; l < nfr; ++l) plan->fdev[f0r + l].role = (l == P.hub) ? 1 : 2;
        f0r += nfr;
      }
    }
    // distributions of Clifford fragments: non-hub ones first (exact
    // distributions a stitched evaluation still forms), hubs after
    {
      long long off = plan->n_dist_nc;
      for (auto& f : plan->fdev)
        if (f.clifford && f.role != 1) { f.dist_off = off; off += (long long)f.nv << f.nA; }
      plan->n_dist_stitch = off;
      for (auto& f : plan->fdev)
        if (f.clifford && f.role == 1) { f.dist_off = off; off += (long long)f.nv << f.nA; }
      for (auto& f : plan->fdev) {
        f.qrow_off = -1;
        if (f.clifford && f.role == 1) {
          f.qrow_off = plan->n_qrows;
          plan->n_qrows += 1ll << (2 * f.n_slots);
          if (f.qout > 4) plan->stitch_ok = false;
        }
      }
    }
    // shot counts: non-hub Clifford fragments first (they are zeroed before
    // sampling), hub fragments after (written whole by the fused sampler)
    {
      long long off = 0;
      for (auto& f : plan->fdev)
        if (f.clifford && f.role != 1) { f.counts_off = off; off += (long long)f.nv << f.nA; }
      plan->n_counts_plain = off;
      for (auto& f : plan->fdev)
        if (f.clifford && f.role == 1) { f.counts_off = off; off += (long long)f.nv << f.nA; }
    }
    std::vector<int2> items_hub, items_plain;
    for (auto& it : items_c) {
      const FragDev& f = plan->fdev[it.x];
      if (f.role == 1) {
        items_hub.push_back(it);
        plan->max_hub_nA = std::max(plan->max_hub_nA, f.nA);
        if (f.m < 2 || f.qout > 4 || f.nA > 16) plan->hub_bytes_ok = false;
      }
      else items_plain.push_back(it);
    }
    plan->n_items_hub = (int)items_hub.size();
    plan->n_items_plain = (int)items_plain.size();
    // fold sets: T of non-hub Clifford fragments (main stream) and non-hub
    // statevector fragments (side branch); T^S of every fragment; then the
    // contraction operands Q (hubs) and T' (the others)
    std::vector<int> fidx_c, fidx_nc, fidx_h, fidx_hn, fidx_o;
    std::vector<long long> tp_c{0}, tp_nc{0}, tp_h{0}, tp_hn{0}, tp_o{0};
    for (int fi = 0; fi < (int)plan->fdev.size(); ++fi) {
      const FragDev& f = plan->fdev[fi];
      const long long t = (1ll << f.m) * (1ll << (2 * f.n_slots));
      const long long tf = f.role == 1 ? 0 : t;    // hubs: T only on request
      if (f.clifford) { fidx_c.push_back(fi); tp_c.push_back(tp_c.back() + tf); }
      else { fidx_nc.push_back(fi); tp_nc.push_back(tp_nc.back() + tf); }
      if (f.role == 1) { fidx_h.push_back(fi); tp_h.push_back(tp_h.back() + t); }
      if (f.role == 1 && !f.clifford) { fidx_hn.push_back(fi); tp_hn.push_back(tp_hn.back() + t); }
      if (f.role == 2) { fidx_o.push_back(fi); tp_o.push_back(tp_o.back() + t); }
    }
    for (auto& P : plan->problems) {
      ProblemDev d{};
      d.k = (int)P.cuts.size();
      d.n_frags = (int)P.frag_ids.size();
      d.frag0 = f0;
      d.hub = P.hub;
      d.n_marg = (int)P.marginal.size();
      d.nz = (int)P.zstrings.size();
      d.marg_off = plan->n_marg;
      d.zexp_off = plan->n_zexp;
      plan->n_marg += 1ll << d.n_marg;
      plan->n_zexp += d.nz;
      plan->out_prefix.push_back(plan->n_marg);
      plan->z_prefix.push_back(plan->n_zexp);
      if (P.hub < 0) {          // not a star: the general contraction over all fragment tensors
        plan->all_star = false;
        d.general = 1;
        d.K = 1ll << (2 * d.k);
      }
      if (P.hub >= 0) {
        const int m_hub = plan->fdev[f0 + P.hub].m;
        d.M = 1 << m_hub;
        d.N = 1 << (d.n_marg - m_hub);
        d.K = 1ll << (2 * d.k);
        auto up4 = [](int x) { return (x + 3) & ~3; };
        d.TN = std::min(up4(d.N), 64);                          // tile: TM x TN, 4x4 per thread,
        d.TM = std::min(up4(d.M), 4096 / d.TN);                 // at most 256 threads
        d.mtiles = (d.M + d.TM - 1) / d.TM;
        d.ntiles = (d.N + d.TN - 1) / d.TN;
        d.hub_T_off = plan->fdev[f0 + P.hub].T_off;
        d.hub_qrow_off = plan->fdev[f0 + P.hub].qrow_off;
        d.tc = (gemm_tc_supported(d.M, d.N, d.K) && d.K >= 4096 && d.M >= 128) ? 1 : 0;
        // leaf by leaf in shared memory, the hub outputs in slices of TM (the
        // contraction never mixes hub outputs), when every intermediate of a
        // slice fits: per hub output the intermediates hold rest_l x N_1..N_l
        // floats (the first leaf reads the hub operand from global memory)
        long long per_m = d.n_frags > 1 ? 1 : d.K, A = 1, rest = d.K;   // the first leaf reads Q^T in place
        int slots = 0;
        for (int l = 0; l < d.n_frags; ++l) {
          if (l == P.hub) continue;
          const FragDev& L = plan->fdev[f0 + l];
          rest >>= 2 * L.n_slots;
          A <<= L.m;
          slots += L.n_slots;
          per_m = std::max(per_m, rest * A);
        }
        auto slice = [&](long long pm) {
          long long t = 1;
          while (2 * t <= d.M && 2 * t * pm <= kDirectSmemFloats && 2 * t + d.N <= kDirectSmemFloats) t *= 2;
          return t;
        };
        long long tm = slice(per_m);
        // staging the operand slice first (coalesced, then every read in shared
        // memory) when that does not shrink the slice
        const long long per_m_staged = std::max(per_m, d.K);
        d.direct_staged = per_m_staged <= kDirectSmemFloats && slice(per_m_staged) == tm;
        if (d.direct_staged) per_m = per_m_staged;
        d.direct = (!d.tc && slots == d.k && per_m <= kDirectSmemFloats && tm + d.N <= kDirectSmemFloats) ? 1 : 0;
        if (d.direct) {
          d.splits = 1;
          d.TM = (int)tm;                      // hub outputs per block
          d.mtiles = (int)(d.M / tm);
          d.r_off = plan->r_total;
          d.part_off = plan->part_total;
          d.blk_off = plan->gemm_blocks;
          for (int t = 0; t < d.mtiles; ++t) plan->direct_items.push_back(make_int2((int)plan->pdev.size(), t));
          plan->direct_stage_floats =
              std::max(plan->direct_stage_floats, std::max(tm * per_m, tm + (long long)d.N));
        }
        if (!d.direct) {
          const long long base = (long long)d.mtiles * d.ntiles;
          const int target = 2 * std::max(c->sm_count, 148);
          const long long max_splits = std::max(1ll, d.K / 32);
          d.splits = (int)std::max(1ll, std::min(max_splits, (target + base - 1) / base));
          // a wide hub operand with few leaf outputs streams through the
          // CUDA-core GEMM (4 hub outputs x N per thread, two CTAs per SM)
          d.stream = (d.N <= 16 && d.M >= 128 && d.M % 4 == 0 && d.K >= 1024 && d.hub_T_off % 4 == 0) ? 1 : 0;
          if (d.stream) {
            d.sthreads = std::min(256, d.M / 4);
            d.smblocks = (d.M / 4 + d.sthreads - 1) / d.sthreads;
            const long long max_ss = std::max(1ll, d.K / 64);
            d.ssplits = (int)std::max(1ll, std::min(max_ss, (long long)(target + d.smblocks - 1) / d.smblocks));
            // the first leaf (lowest leaf-output bits) with 1-4 cuts and 1-2 marginal bits
            // is contracted while streaming
            int l1 = 0;
            while (l1 < d.n_frags && l1 == P.hub) ++l1;
            if (l1 < d.n_frags) {
              const FragDev& L = plan->fdev[f0 + l1];
              const int N1 = 1 << L.m, G1 = 1 << (2 * L.n_slots);
              // (large operands only: a small star's two extra launches cost more than its FMAs)
              if (L.n_slots >= 1 && L.n_slots <= 2 && N1 <= 2 && d.N % N1 == 0 && d.N / N1 >= 1 &&
                  d.K * (long long)d.M >= (1ll << 24)) {
                d.fact = 1;
                d.fl1 = l1;
                d.fl1_T_off = L.T_off;
                d.G1 = G1;
                d.N1 = N1;
                d.NR = d.N / N1;
                d.ndig1 = L.n_slots;
                for (int i = 0; i < L.n_slots; ++i) d.dig1[i] = L.slot_cut[i];
                d.ndigr = 0;
                for (int cc = 0; cc < d.k; ++cc) {
                  bool mine = false;
                  for (int i = 0; i < L.n_slots; ++i) mine = mine || L.slot_cut[i] == cc;
                  if (!mine) d.digr[d.ndigr++] = cc;
                }
              }
            }
          }
          plan->chain = 1;
          d.r_off = plan->r_total;
          plan->r_total += d.K * d.N;
          d.part_off = (plan->part_total + 3) & ~3ll;      // float4 stores of the streaming GEMM
          plan->part_total = d.part_off + (long long)std::max(d.splits, d.stream ? d.ssplits : 0) * d.M * d.N;
          d.blk_off = plan->gemm_blocks;
          plan->gemm_blocks += base * d.splits;
          plan->max_tile_smem = std::max(plan->max_tile_smem, 16 * (d.TM + d.TN) * 4);
        }
        if (d.tc) {
          d.rt_off = (plan->rt_total + 63) & ~63ll;
          plan->rt_total = d.rt_off + d.K * d.N;
        }
      }
      plan->r_prefix.push_back(plan->r_total);
      plan->blk_prefix.push_back(plan->gemm_blocks);
      f0 += d.n_frags;
      plan->pdev.push_back(d);
    }

    // the scratch holds every problem's R operand first, then the split-K partials
    plan->r_total = (plan->r_total + 3) & ~3ll;
    for (auto& d : plan->pdev) d.part_off += plan->r_total;
    std::vector<CliffordOp> prep(4), basis(3);
    std::vector<float> prepm(32), basism(24);
    for (int s = 0; s < 4; ++s) { prep[s] = prep_op(s); prep_matrix(s, &prepm[8 * s]); }
    for (int b = 0; b < 3; ++b) { basis[b] = basis_op(b); basis_matrix(b, &basism[8 * b]); }

    int *d_fidx_c, *d_fidx_nc, *d_fidx_h, *d_fidx_hn, *d_fidx_o;
    long long *d_tp_c, *d_tp_nc, *d_tp_h, *d_tp_hn, *d_tp_o;
    if (!c->host_only) {
      Staging st;
      st.add(fidx_c, &d_fidx_c); st.add(fidx_nc, &d_fidx_nc); st.add(tp_c, &d_tp_c);
      st.add(tp_nc, &d_tp_nc); st.add(fidx_h, &d_fidx_h); st.add(fidx_o, &d_fidx_o);
      st.add(tp_h, &d_tp_h); st.add(tp_o, &d_tp_o);
      st.add(fidx_hn, &d_fidx_hn); st.add(tp_hn, &d_tp_hn);
      st.add(items_hub, &plan->d_items_hub); st.add(items_plain, &plan->d_items_plain);
      bool okf = st.commit(c, plan->A);
      if (!okf) { return fail(c, CCS_ERR_OOM, "plan upload failed"); }
      plan->fold_cliff = FoldSet{d_fidx_c, d_tp_c, (int)fidx_c.size(), tp_c.back()};
      plan->fold_nc = FoldSet{d_fidx_nc, d_tp_nc, (int)fidx_nc.size(), tp_nc.back()};
      plan->fold_hubs = FoldSet{d_fidx_h, d_tp_h, (int)fidx_h.size(), tp_h.back()};
      plan->fold_hubs_nc = FoldSet{d_fidx_hn, d_tp_hn, (int)fidx_hn.size(), tp_hn.back()};
      plan->fold_others = FoldSet{d_fidx_o, d_tp_o, (int)fidx_o.size(), tp_o.back()};
    }
    if (c->host_only) {
      plan->dp.n_items_cliff = (int)items_c.size();
      plan->dp.n_items_nc = (int)items_nc.size();
      *out = owned.release();
      return CCS_OK;
    }
    DevPlan& dp = plan->dp;
    FragDev* dfr; CliffordOp* dco; NCOp* dno; int* dmo; int* dwi; int* dzo; int2* dic; int2* din; int2* dib; int* dcf;
    int2* diz = nullptr; int2* dzb = nullptr; int2* dip = nullptr;
    ProblemDev* dpr; CliffordOp* dpo; CliffordOp* dbo; float* dpm; float* dbm;
    Staging st;
    st.add(plan->fdev, &dfr); st.add(cops, &dco); st.add(nops, &dno); st.add(moments, &dmo); st.add(wires, &dwi);
    st.add(zoffs, &dzo); st.add(items_c, &dic); st.add(items_nc, &din); st.add(items_b, &dib);
    st.add(cliff_frags, &dcf); st.add(items_z, &diz); st.add(items_p, &dip); st.add(zblocks, &dzb); st.add(plan->pdev, &dpr); st.add(prep, &dpo); st.add(basis, &dbo);
    st.add(prepm, &dpm); st.add(basism, &dbm); st.add(plan->t_prefix, &plan->d_t_prefix);
    st.add(plan->out_prefix, &plan->d_out_prefix);
    st.add(plan->z_prefix, &plan->d_z_prefix); st.add(plan->r_prefix, &plan->d_r_prefix);
    st.add(plan->blk_prefix, &plan->d_blk_prefix); st.add(plan->direct_items, &plan->d_direct_items);
    bool ok = st.commit(c, plan->A);
    if (!ok) { return fail(c, CCS_ERR_OOM, "plan upload failed"); }
    dp.frags = dfr; dp.cops = dco; dp.nops = dno; dp.moments = dmo; dp.wires = dwi; dp.zoffs = dzo;
    dp.items_cliff = dic; dp.items_nc = din; dp.nc_basis_chunk = plan->nc_basis_chunk;
    dp.n_items_cliff = (int)items_c.size(); dp.n_items_nc = (int)items_nc.size();
    dp.items_body = dib; dp.n_items_body = (int)items_b.size(); dp.max_body_cols = max_body_cols;
    dp.cliff_frags = dcf; dp.n_cliff_frags = (int)cliff_frags.size();
    dp.items_zimg = diz; dp.n_items_zimg = (int)items_z.size();
    dp.items_proj = dip; dp.n_items_proj = (int)items_p.size();
    dp.zblocks = dzb; dp.n_zblocks = (int)zblocks.size();
    dp.body_words_max = body_words_max; dp.img_words_max = img_words_max;
    dp.max_body_stage_words = max_body_stage;
    dp.max_moment_ops = max_moment_ops;
    dp.problems = dpr; dp.n_problems = (int)plan->pdev.size();
    dp.prep_ops = dpo; dp.basis_ops = dbo; dp.prep_mats = dpm; dp.basis_mats = dbm;
    // the plan's arrays are on the device before it is handed out (it may be
    // used from another context's stream); other work on the stream is not waited for
    if (!Staging::upload_wait(c)) { return fail(c, CCS_ERR_CUDA, "plan upload"); }
    *out = owned.release();
    return CCS_OK;
  });
}

void ccs_plan_free(ccs_plan p) { delete p; }

int ccs_cut_candidates(ccs_ctx c, const ccs_problem* q, const ccs_cut_opts* opts, ccs_cut* cuts_out,
                       int cap_cuts, int* offsets, double* costs, int cap_cands) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !q || !cuts_out || !offsets || cap_cands < 1) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    ccs_cut_opts o{kMaxCuts, 10, 0};
    if (opts) o = *opts;
    Problem P;
    P.n_qubits = q->n_qubits;
    std::string err;
    int rc = check_circuit(*q, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    rc = load_gates(q->gates, q->n_gates, P.gates, P.gparam, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    P.marginal.assign(q->marginal, q->marginal + q->n_marginal);
    CutSearchOpts so;
    so.max_cuts = std::min(o.max_cuts, kMaxCuts);
    so.max_nc_width = std::min(o.max_nc_width > 0 ? o.max_nc_width : 10, kMaxNCWidth);
    std::vector<CutCandidate> cands;
    rc = greedy_cuts(P, so, cands, err);
    if (rc != CCS_OK) return fail(c, rc, err);
    int n = 0, used = 0;
    offsets[0] = 0;
    for (auto& cd : cands) {
      if (n >= cap_cands || used + (int)cd.cuts.size() > cap_cuts) break;
      for (auto& x : cd.cuts) cuts_out[used++] = x;
      if (costs) costs[n] = cd.cost;
      offsets[++n] = used;
    }
    return n;
  });
}

// Evaluation as two branches: Clifford variants (tableaus -> spaces/Z-values
// -> sampling -> fold) on the context stream, statevector variants (+ their
// fold) on the side stream, forked after the memsets and joined at the end.
// With profiling on, everything runs on the context stream so each stage's
// events bracket one kernel.
static int enqueue_eval(ccs_ctx c, ccs_plan p, ccs_res r) {
  cudaStream_t s = c->stream;
  const EvalParams& e = r->ep;
  cudaError_t err;
  if ((err = cudaMemsetAsync(r->dr.work, 0, (4 + (size_t)p->dp.n_cliff_frags) * sizeof(unsigned), s)) != cudaSuccess)
    return cuda_fail(c, err, "memset");
  if (e.mode == CCS_SAMPLED && p->n_counts_plain)
    if ((err = cudaMemsetAsync(r->dr.counts, 0, p->n_counts_plain * sizeof(uint32_t), s)) != cudaSuccess)
      return cuda_fail(c, err, "memset counts");
  if (e.mode == CCS_EXACT && p->n_dist)
    if ((err = cudaMemsetAsync(r->dr.dist, 0, p->n_dist * sizeof(float), s)) != cudaSuccess)
      return cuda_fail(c, err, "memset dist");
  if (e.mode == CCS_STITCH && p->n_dist_stitch > p->n_dist_nc)    // the non-hub Clifford distributions
    if ((err = cudaMemsetAsync(r->dr.dist + p->n_dist_nc, 0, (p->n_dist_stitch - p->n_dist_nc) * sizeof(float),
                               s)) != cudaSuccess)
      return cuda_fail(c, err, "memset dist");
  const DevPlan& dp = p->dp;
  const bool fork = dp.n_items_nc > 0 && !c->profiling;
  cudaStream_t s2 = fork ? c->side : s;
  if (fork) {
    if ((err = cudaEventRecord(c->fork_ev, s)) != cudaSuccess) return cuda_fail(c, err, "fork");
    if ((err = cudaStreamWaitEvent(s2, c->fork_ev, 0)) != cudaSuccess) return cuda_fail(c, err, "fork wait");
  }
  if (dp.n_items_nc) {
    int grid = std::min(dp.n_items_nc, c->sm_count * 4);
    int threads = std::min(512, std::max(32, 1 << p->max_nc_n));   // one output amplitude per thread
    stage_begin(c, ST_STATEVEC);
    if ((err = launch_statevector(dp, r->dr, p->max_nc_n, threads, grid, s2)) != cudaSuccess)
      return cuda_fail(c, err, "statevector kernel");
    stage_end(c, ST_STATEVEC);
    if ((err = launch_fold(dp, r->dr, e, p->fold_nc, s2)) != cudaSuccess) return cuda_fail(c, err, "fold kernel");
  }
  if (dp.n_items_cliff) {
    const int threads = r->cliff_threads;
    const int smem_words = e.shared_body ? p->body_smem_words : p->cliff_smem_words;
    const size_t smem = (size_t)smem_words * 8;
    int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2048 / threads, (c->smem_optin + 1024) / (smem + 2048)));
    int grid = std::min(dp.n_items_cliff, c->sm_count * per_sm);
    stage_begin(c, ST_CLIFFORD);
    if (e.shared_body) {
      if ((err = launch_body(dp, r->dr, (int)c->smem_optin, e.screen != 0, s)) != cudaSuccess)
        return cuda_fail(c, err, "body kernel");
      if (e.screen && (err = launch_screen(dp, r->dr, e, c->sm_count, (int)c->smem_optin, s)) != cudaSuccess)
        return cuda_fail(c, err, "screen kernel");
    }
    if (!e.screen &&
        (err = launch_clifford(dp, r->dr, e, threads, e.shared_body ? 1 : r->cliff_words, smem_words, grid, s)) !=
            cudaSuccess)
      return cuda_fail(c, err, "clifford kernel");
    stage_end(c, ST_CLIFFORD);
    if (e.mode == CCS_SAMPLED) {
      stage_begin(c, ST_SAMPLE);
      if ((err = launch_sample_hub(dp, r->dr, e, p->d_items_hub, p->n_items_hub, p->max_hub_nA, r->hub_threads,
                                   e.keep_tableaus, p->hub_bytes_ok && r->hub_bytes,
                                   s)) != cudaSuccess)
        return cuda_fail(c, err, "hub sample kernel");
      if ((err = launch_sample(dp, r->dr, e, p->d_items_plain, p->n_items_plain, r->sample_spc, 256, s)) !=
          cudaSuccess)
        return cuda_fail(c, err, "sample kernel");
      stage_end(c, ST_SAMPLE);
    }
    if (e.mode == CCS_STITCH) {   // Clifford hubs: the operand in closed form from the outcome spaces
      stage_begin(c, ST_SAMPLE);
      if ((err = launch_hub_exact(dp, r->dr, p->d_items_hub, p->n_items_hub, s)) != cudaSuccess)
        return cuda_fail(c, err, "hub exact kernel");
      stage_end(c, ST_SAMPLE);
    }
    stage_begin(c, ST_FOLD);
    if ((err = launch_fold(dp, r->dr, e, p->fold_cliff, s)) != cudaSuccess) return cuda_fail(c, err, "fold kernel");
    stage_end(c, ST_FOLD);
  }
  if (fork) {
    if ((err = cudaEventRecord(c->join_ev, s2)) != cudaSuccess) return cuda_fail(c, err, "join");
    if ((err = cudaStreamWaitEvent(s, c->join_ev, 0)) != cudaSuccess) return cuda_fail(c, err, "join wait");
  }
  stage_begin(c, ST_OPERANDS);
  // hubs: Clifford hubs in sampled and stitched modes already have Q (the
  // fused sampler, the closed form)
  const FoldSet& hubs = e.mode == CCS_EXACT ? p->fold_hubs : p->fold_hubs_nc;
  if ((err = launch_operands(dp, r->dr, e, hubs, p->fold_others, s)) != cudaSuccess)
    return cuda_fail(c, err, "operand kernels");
  stage_end(c, ST_OPERANDS);
  return CCS_OK;
}

// Autotuner: time every (Clifford threads per CTA, shots per sampler CTA)
// candidate on this plan with CUDA events (one warm-up + three timed
// evaluations each) and keep the fastest; cached per shape bucket (widest
// Clifford fragment rounded up to 64 wires, Clifford variant count rounded up
// to a power of two, shots, mode).
constexpr int kVariantPathMaxItems = 8192;   // Clifford variants up to which the autotuner also times the per-variant path

static int autotune(ccs_ctx c, ccs_plan p, ccs_res r) {
  int max_n = 0;
  for (auto& f : p->fdev)
    if (f.clifford) max_n = std::max(max_n, f.n);
  int items = 1;
  while (items < p->dp.n_items_cliff) items <<= 1;
  const auto key =
      std::make_tuple((max_n + 63) / 64, items, r->ep.shots, r->ep.mode * 4 + r->ep.shared_body * 2 + r->ep.screen);
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) {
    int vp = 0;
    std::tie(r->cliff_threads, r->cliff_words, r->sample_spc, r->hub_threads, vp) = it->second;
    r->hub_bytes = r->hub_threads < 0;       // cached as minus the threads of the byte-counter kernel
    r->hub_threads = std::abs(r->hub_threads);
    r->variant_path = vp != 0;
    if (r->variant_path) { r->ep.shared_body = 0; r->ep.screen = 0; }
    return CCS_OK;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, CCS_ERR_CUDA, "autotune events");
  // one warm-up and three timed evaluations of the current shape
  auto time_it = [&](float* ms) -> int {
    int rc = enqueue_eval(c, p, r);
    if (rc != CCS_OK) return rc;
    cudaEventRecord(e0, c->stream);
    for (int rep = 0; rep < 3 && rc == CCS_OK; ++rep) rc = enqueue_eval(c, p, r);
    cudaEventRecord(e1, c->stream);
    if (rc != CCS_OK) return rc;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return fail(c, CCS_ERR_CUDA, "autotune timing");
    return CCS_OK;
  };
  // coordinate descent: tableau CTA shape, then plain-sampler chunk, then hub-sampler CTA
  const int threads_c[] = {128, 256, 512};
  const int words_c[] = {1, 2, 4, 8};
  const int spc_c[] = {1024, 2048, 4096, 8192};
  const int hub_c[] = {128, 512, 256, 512};  // 16-bit counters, then byte counters
  const int max_w = 2 * ((max_n + 63) / 64);
  const bool sampled = r->ep.mode == CCS_SAMPLED;
  int rc = CCS_OK;
  float best = 1e30f, ms = 0.f;
  int bt = r->cliff_threads, bw = r->cliff_words, bs = r->sample_spc, bh = r->hub_threads;
  // (the tableau kernel does not run after the screen: one baseline timing)
  const int n_ti = r->ep.screen ? 1 : 3;
  for (int ti = 0; ti < n_ti && rc == CCS_OK; ++ti)
    for (int wi = 0; wi < 4 && rc == CCS_OK; ++wi) {
      if (words_c[wi] > max_w || (r->ep.shared_body && words_c[wi] != 1)) continue;
      if (r->ep.screen) { if ((rc = time_it(&ms)) == CCS_OK) best = ms; break; }
      r->cliff_threads = threads_c[ti];
      r->cliff_words = words_c[wi];
      if ((rc = time_it(&ms)) == CCS_OK && ms < best) { best = ms; bt = threads_c[ti]; bw = words_c[wi]; }
    }
  r->cliff_threads = bt;
  r->cliff_words = bw;
  for (int si = 0; sampled && p->n_items_plain && si < 4 && rc == CCS_OK; ++si) {
    r->sample_spc = spc_c[si];
    if ((rc = time_it(&ms)) == CCS_OK && ms < best) { best = ms; bs = spc_c[si]; }
  }
  r->sample_spc = bs;
  bool bb = r->hub_bytes;
  for (int hi = 0; sampled && p->n_items_hub && hi < 4 && rc == CCS_OK; ++hi) {
    const bool bytes = hi >= 2;
    if (bytes && !p->hub_bytes_ok) continue;
    r->hub_bytes = bytes;
    r->hub_threads = hub_c[hi];
    if ((rc = time_it(&ms)) == CCS_OK && ms < best) { best = ms; bh = hub_c[hi]; bb = bytes; }
  }
  r->hub_threads = bh;
  r->hub_bytes = bb;
  // Small plans whose tableaus fit in shared memory: the per-variant path
  // (every variant simulates its whole circuit in one kernel, no shared-body
  // chain) can be faster than the shared body's chain of short kernels; it
  // is timed with its own tableau CTA shapes and kept if faster.  Both paths
  // give the same outcome spaces, shots and values.
  r->variant_path = false;
  if (rc == CCS_OK && r->ep.shared_body && r->ep.screen && p->tableau_fits && p->dp.n_items_cliff > 0 &&
      p->dp.n_items_cliff <= kVariantPathMaxItems) {
    if ((rc = time_it(&ms)) == CCS_OK) best = ms;      // the tuned shared-body path
    float best_v = 1e30f;
    int vt = bt, vw = bw;
    r->ep.shared_body = 0;
    r->ep.screen = 0;
    for (int ti = 0; ti < 3 && rc == CCS_OK; ++ti)
      for (int wi = 0; wi < 4 && rc == CCS_OK; ++wi) {
        if (words_c[wi] > max_w) continue;
        r->cliff_threads = threads_c[ti];
        r->cliff_words = words_c[wi];
        if ((rc = time_it(&ms)) == CCS_OK && ms < best_v) { best_v = ms; vt = threads_c[ti]; vw = words_c[wi]; }
      }
    if (rc == CCS_OK && best_v < best) {
      r->variant_path = true;
      bt = vt;
      bw = vw;
    } else {
      r->ep.shared_body = 1;
      r->ep.screen = 1;
    }
    r->cliff_threads = bt;
    r->cliff_words = bw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CCS_OK) return rc;
  c->tuned[key] = std::make_tuple(bt, bw, bs, bb ? -bh : bh, r->variant_path ? 1 : 0);
  return CCS_OK;
}

int ccs_get_tuning(ccs_ctx c, ccs_res r, int* cliff_threads, int* words_per_op, int* shots_per_cta,
                   int* hub_threads, int* variant_path) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !r) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (hub_threads) *hub_threads = (r->hub_bytes && r->plan->hub_bytes_ok) ? -r->hub_threads : r->hub_threads;
    if (variant_path) *variant_path = r->ep.shared_body ? 0 : 1;
    if (cliff_threads) *cliff_threads = r->cliff_threads;
    if (words_per_op) *words_per_op = r->ep.shared_body ? 1 : r->cliff_words;
    if (shots_per_cta) *shots_per_cta = r->sample_spc;
    return CCS_OK;
  });
}

int ccs_eval_variants(ccs_ctx c, ccs_plan p, const ccs_eval_opts* opts, ccs_res* res) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !p || !opts || !res) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (opts->mode != CCS_EXACT && opts->mode != CCS_SAMPLED && opts->mode != CCS_STITCH)
      return fail(c, CCS_ERR_INVALID_ARG, "bad mode");
    if ((opts->keep_tableaus || opts->per_variant_body) && !p->tableau_fits)
      return fail(c, CCS_ERR_UNSUPPORTED, "a Clifford fragment's tableau does not fit in shared memory "
                                          "(kept tableaus and per-variant bodies need it; at most 640 wires)");
    if (opts->mode == CCS_STITCH && !p->stitch_ok)
      return fail(c, CCS_ERR_UNSUPPORTED, "stitched mode: a Clifford hub with more than 4 quantum outputs");
    if (opts->mode == CCS_SAMPLED && opts->shots == 0) return fail(c, CCS_ERR_INVALID_ARG, "zero shots");
    if (opts->mode == CCS_SAMPLED && opts->shots > 0xffffu && p->max_hub_nA > 15)
      return fail(c, CCS_ERR_UNSUPPORTED, "more than 65535 shots with a 16-bit hub outcome space");
    if (opts->mode == CCS_SAMPLED && p->max_hub_nA > 16)   // the hub histogram lives in shared memory
      return fail(c, CCS_ERR_UNSUPPORTED, "hub measured set wider than 16 bits in sampled mode");
    if (c->host_only) return fail(c, CCS_ERR_UNSUPPORTED, "host-only context cannot evaluate");
    cudaSetDevice(c->device);
    ccs_res r = *res;
    if (r && r->plan != p) return fail(c, CCS_ERR_INVALID_ARG, "result belongs to another plan");
    if (!r) {
      std::unique_ptr<ccs_res_s> owned_r(new ccs_res_s());   // freed on a failed allocation or an exception
      r = owned_r.get();
      r->plan = p;
      r->A.ctx = c;
      DevRes& d = r->dr;
      d.spaces = r->A.get<SpaceRec>(std::max<long long>(p->n_spaces, 1));
      d.dist = r->A.get<float>(std::max<long long>(p->n_dist_nc, 1));   // exact / stitched modes widen it
      r->dist_len = p->n_dist_nc;
      d.qnz = r->A.get<uint8_t>(std::max<long long>(p->n_qrows, 1));
      d.zval = r->A.get<float>(std::max<long long>(p->n_zval, 1));
      d.T = r->A.get<float>(std::max<long long>(p->n_T, 1));
      d.TQ = r->A.get<float>(std::max<long long>(p->n_T, 1));
      d.marg = r->A.get<double>(std::max<long long>(p->n_marg, 1));
      d.zexp = r->A.get<double>(std::max<long long>(p->n_zexp, 1));
      d.work = r->A.get<unsigned>(4 + (long long)p->dp.n_cliff_frags);   // + per-fragment record counters
      d.fragcnt = d.work ? d.work + 4 : nullptr;
      d.body = r->A.get<unsigned long long>(std::max<long long>(p->n_body, 2));
      d.rowbasis = r->A.get<unsigned long long>(std::max<long long>((long long)kRowBasisWords * p->dp.n_cliff_frags, 1));
      d.zimg = r->A.get<unsigned long long>(std::max<long long>(p->n_zimg, 1));
      d.pbasis = r->A.get<uint32_t>(std::max<long long>(p->n_pbasis, 1));

      d.status = r->A.get<unsigned>(4);
      r->scratch = r->A.get<float>(std::max<long long>(p->r_total + p->part_total, 1));
      {   // default launch shape before any tuning: wide tableaus take 8 words per op, 512 threads
        int max_n = 0;
        for (auto& f : p->fdev)
          if (f.clifford) max_n = std::max(max_n, f.n);
        const int W = 2 * ((max_n + 63) / 64);
        r->cliff_words = W >= 16 ? 8 : W >= 8 ? 4 : 1;
        r->cliff_threads = max_n > 256 ? 512 : 256;
        // small hub CTAs when a variant has few shots and few outputs (more CTAs per SM);
        // byte counters when the histogram would otherwise fill an SM's shared memory
        r->hub_bytes = p->hub_bytes_ok && p->max_hub_nA >= 13;
        r->hub_threads = r->hub_bytes ? 256 : (p->max_hub_nA <= 12 && opts->shots <= 4096) ? 128 : 512;
      }
      if (p->rt_total) {
        d.TQh = r->A.get<uint16_t>(p->n_T);
        r->rt_scratch = r->A.get<uint16_t>(p->rt_total);
      }
      if (!d.spaces || !d.dist || !d.qnz || !d.zval || !d.T || !d.TQ || !d.marg || !d.zexp || !d.work || !d.status ||
          !d.body || !d.rowbasis || !d.zimg || !d.fragcnt || !d.pbasis ||
          !r->scratch || (p->rt_total && (!d.TQh || !r->rt_scratch))) {
        return fail(c, CCS_ERR_OOM, "result allocation failed");
      }
      cudaMemsetAsync(d.status, 0, 4 * sizeof(unsigned), c->stream);
      *res = owned_r.release();
    }
    // buffers a mode needs are added on first use; a replaced buffer drops the captured graph
    auto drop_graph = [&]() {
      if (r->graph) { cudaGraphExecDestroy(r->graph); r->graph = nullptr; }
    };
    const bool want_full_counts = opts->keep_tableaus && p->n_counts > p->n_counts_plain;
    if (opts->mode == CCS_SAMPLED && p->n_counts && (!r->have_counts || (want_full_counts && !r->counts_full))) {
      r->dr.counts = r->A.get<uint32_t>(want_full_counts ? p->n_counts : std::max<long long>(p->n_counts_plain, 1));
      if (!r->dr.counts) return fail(c, CCS_ERR_OOM, "counts allocation failed");
      r->have_counts = true;
      r->counts_full = want_full_counts;
      drop_graph();
    }
    {
      const long long need = opts->mode == CCS_EXACT ? p->n_dist : opts->mode == CCS_STITCH ? p->n_dist_stitch
                                                                                          : p->n_dist_nc;
      if (need > r->dist_len) {
        float* nd = r->A.get<float>(need);   // every evaluation rewrites what it reads
        if (!nd) return fail(c, CCS_ERR_OOM, "distribution allocation failed");
        r->dr.dist = nd;
        r->dist_len = need;
        drop_graph();
      }
    }
    if (opts->keep_tableaus && !r->have_tabs && p->n_tab) {
      r->dr.tabs = r->A.get<unsigned long long>(p->n_tab);
      if (!r->dr.tabs) return fail(c, CCS_ERR_OOM, "tableau allocation failed");
      r->have_tabs = true;
    }
    EvalParams e{};
    e.mode = opts->mode;
    e.shots = opts->mode == CCS_SAMPLED ? opts->shots : 0;
    e.seed_lo = opts->seed_lo;
    e.seed_hi = opts->seed_hi;
    for (int rd = 0; rd < 10; ++rd) {
      e.keys.k[rd][0] = e.seed_lo + (uint32_t)rd * 0x9E3779B9u;
      e.keys.k[rd][1] = e.seed_hi + (uint32_t)rd * 0xBB67AE85u;
    }
    e.keep_tableaus = opts->keep_tableaus && r->have_tabs;
    // the autotuner's path choice holds for later default-path calls on this result
    const bool variant_path = r->variant_path && !opts->keep_tableaus && p->tableau_fits;
    e.shared_body = (opts->per_variant_body || variant_path) ? 0 : 1;
    e.screen = e.shared_body && p->dp.n_cliff_frags > 0 && !e.keep_tableaus;
    if (opts->hub_sampler < 0 || opts->hub_sampler > 3) return fail(c, CCS_ERR_INVALID_ARG, "bad hub sampler");
    e.hub_sampler = opts->hub_sampler;
    if (opts->hub_sampler == 1) {
      r->hub_bytes = false;
      if (r->hub_threads != 128) r->hub_threads = 512;
    }
    if (opts->hub_sampler >= 2) {
      r->hub_bytes = p->hub_bytes_ok;
      r->hub_threads = opts->hub_sampler == 3 ? 512 : 256;
    }
    e.inv_shots = e.shots ? 1.0 / (double)e.shots : 0.0;
    r->ep = e;
    {   // sampled hubs keep exact 16-bit count sums (|sum| <= shots)
      const int i16 = (e.mode == CCS_SAMPLED && e.shots <= 32767u) ? 1 : 0;
      if (i16 != r->eval_i16) drop_graph();
      r->eval_i16 = i16;
      r->dr.hub_i16 = i16;   // a maximum-likelihood correction may have left the operand in FP32
      r->ml_applied = 0;
      r->dr.hub_scale = (float)e.inv_shots;
    }
    if (opts->autotune && !r->graph && opts->hub_sampler == 0) {
      const bool prof = c->profiling;
      c->profiling = false;
      int rc = autotune(c, p, r);
      c->profiling = prof;
      if (rc != CCS_OK) return rc;
      e = r->ep;                             // the autotuner may have chosen the per-variant path
    }
    if (!opts->use_graph || c->profiling) {
      c->stage_mask = 0;
      return enqueue_eval(c, p, r);
    }
    const bool same = r->graph && r->graph_key.mode == e.mode && r->graph_key.shots == e.shots &&
                      r->graph_key.seed_lo == e.seed_lo && r->graph_key.seed_hi == e.seed_hi &&
                      r->graph_key.keep_tableaus == e.keep_tableaus && r->graph_key.shared_body == e.shared_body &&
                      r->graph_key.hub_sampler == e.hub_sampler;
    if (!same) {
      if (r->graph) { cudaGraphExecDestroy(r->graph); r->graph = nullptr; }
      cudaStream_t s = c->stream;
      bool tmp_stream = false;
      if (s == nullptr) {   // the legacy stream cannot be captured
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(c, CCS_ERR_CUDA, "stream");
        tmp_stream = true;
      }
      cudaStream_t saved = c->stream;
      c->stream = s;
      cudaGraph_t g;
      cudaError_t err = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (err != cudaSuccess) { c->stream = saved; return cuda_fail(c, err, "begin capture"); }
      const long long before = launch_count();
      int rc = enqueue_eval(c, p, r);
      r->graph_launches = launch_count() - before;
      note_launches(-r->graph_launches);      // captured, not launched
      err = cudaStreamEndCapture(s, &g);
      c->stream = saved;
      if (tmp_stream) cudaStreamDestroy(s);
      if (rc != CCS_OK) return rc;
      if (err != cudaSuccess) return cuda_fail(c, err, "end capture");
      err = cudaGraphInstantiate(&r->graph, g, 0);
      cudaGraphDestroy(g);
      if (err != cudaSuccess) return cuda_fail(c, err, "graph instantiate");
      r->graph_key = e;
    }
    cudaError_t err = cudaGraphLaunch(r->graph, c->stream);
    if (err != cudaSuccess) return cuda_fail(c, err, "graph launch");
    note_launches(r->graph_launches);
    return CCS_OK;
  });
}

void ccs_res_free(ccs_res r) { delete r; }

static int check_status(ccs_ctx c, ccs_res r) {
  unsigned st[4];
  cudaError_t e = cudaMemcpyAsync(st, r->dr.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  if (st[0]) return fail(c, CCS_ERR_DEVICE_CHECK, "device consistency check failed (code " + std::to_string(st[0]) + ")");
  return CCS_OK;
}

int ccs_recombine(ccs_ctx c, ccs_plan p, ccs_res r, const ccs_recomb_opts* opts, double* marginal_out,
                  double* zexp_out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !p || !r || r->plan != p) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (c->host_only) return fail(c, CCS_ERR_UNSUPPORTED, "host-only context cannot recombine");
    const int prec = opts ? opts->precision : CCS_FP32;
    const bool on_dev = opts && opts->outputs_on_device;
    if (prec != CCS_FP32 && prec != CCS_BF16) return fail(c, CCS_ERR_INVALID_ARG, "bad precision");
    cudaSetDevice(c->device);
    const bool stitched = r->ep.mode == CCS_STITCH;
    const bool tc = !(opts && opts->no_tensor_cores) && !stitched;   // stitched rows skip zeros on CUDA cores
    RecombSizes rz{p->r_total, p->part_total, p->gemm_blocks, p->n_marg, p->n_zexp,
                   p->d_direct_items, (int)p->direct_items.size(), (int)p->direct_stage_floats, p->chain,
                   p->d_r_prefix, p->d_blk_prefix, p->d_out_prefix, p->d_z_prefix, p->max_tile_smem,
                   p->pdev.data(), (int)p->pdev.size(), r->rt_scratch, tc ? 1 : 0, stitched ? 1 : 0, KRange{0, -1},
                   p->all_star ? 0 : 1};
    if (opts && (opts->k_lo || opts->k_hi)) {
      if (opts->k_hi && opts->k_hi <= opts->k_lo) return fail(c, CCS_ERR_INVALID_ARG, "empty cut-index range");
      if (opts->k_lo > (1ull << 62) || opts->k_hi > (1ull << 62)) return fail(c, CCS_ERR_INVALID_ARG, "bad range");
      rz.krange = KRange{(long long)opts->k_lo, opts->k_hi ? (long long)opts->k_hi : -1};
    }
    cudaError_t e;
    if (opts && opts->use_graph && !c->profiling && rz.krange.full()) {
      const int key = prec * 2 + (tc ? 1 : 0) + (stitched ? 4 : 0) + (r->dr.hub_i16 ? 8 : 0);
      if (!r->rgraph || r->rgraph_key != key) {
        if (r->rgraph) { cudaGraphExecDestroy(r->rgraph); r->rgraph = nullptr; }
        cudaStream_t s = c->stream;
        bool tmp_stream = false;
        if (s == nullptr) {   // the legacy stream cannot be captured
          if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(c, CCS_ERR_CUDA, "stream");
          tmp_stream = true;
        }
        cudaGraph_t g;
        if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
          if (tmp_stream) cudaStreamDestroy(s);
          return cuda_fail(c, e, "begin capture");
        }
        const long long before = launch_count();
        cudaError_t le = launch_recombine(p->dp, r->dr, prec, rz, r->scratch, r->dr.marg, r->dr.zexp, s);
        r->rgraph_launches = launch_count() - before;
        note_launches(-r->rgraph_launches);      // captured, not launched
        e = cudaStreamEndCapture(s, &g);
        if (tmp_stream) cudaStreamDestroy(s);
        if (le != cudaSuccess) return cuda_fail(c, le, "recombine kernel");
        if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
        e = cudaGraphInstantiate(&r->rgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
        r->rgraph_key = key;
      }
      if ((e = cudaGraphLaunch(r->rgraph, c->stream)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
      note_launches(r->rgraph_launches);
    } else {
      stage_begin(c, ST_RECOMB);
      e = launch_recombine(p->dp, r->dr, prec, rz, r->scratch, r->dr.marg, r->dr.zexp, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "recombine kernel");
      stage_end(c, ST_RECOMB);
    }
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (marginal_out && p->n_marg)
      if ((e = cudaMemcpyAsync(marginal_out, r->dr.marg, p->n_marg * sizeof(double), kind, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "copy marginal");
    if (zexp_out && p->n_zexp)
      if ((e = cudaMemcpyAsync(zexp_out, r->dr.zexp, p->n_zexp * sizeof(double), kind, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "copy zexp");
    if (on_dev) return CCS_OK;
    return check_status(c, r);
  });
}

// --- inspection -------------------------------------------------------------
static const Frag* find_frag(ccs_plan p, int problem, int fragment, int* global) {
  if (problem < 0 || problem >= (int)p->problems.size()) return nullptr;
  const Problem& P = p->problems[problem];
  if (fragment < 0 || fragment >= (int)P.frag_ids.size()) return nullptr;
  *global = P.frag_ids[fragment];
  return &p->frags[*global];
}

int ccs_plan_counts(ccs_ctx c, ccs_plan p, int problem, int* nf, int* nc) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!p || problem < 0 || problem >= (int)p->problems.size()) return fail(c, CCS_ERR_INVALID_ARG, "bad problem");
    if (nf) *nf = (int)p->problems[problem].frag_ids.size();
    if (nc) *nc = (int)p->problems[problem].cuts.size();
    return CCS_OK;
  });
}

int ccs_fragment_info_get(ccs_ctx c, ccs_plan p, int problem, int fragment, ccs_fragment_info* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    int g;
    const Frag* f = p ? find_frag(p, problem, fragment, &g) : nullptr;
    if (!f || !out) return fail(c, CCS_ERR_INVALID_ARG, "bad fragment");
    out->n_wires = f->n();
    out->clifford = f->clifford;
    out->n_variants = f->n_variants();
    out->n_qin = (int)f->qin_wire.size();
    out->n_qout = (int)f->qout_wire.size();
    out->n_marg = (int)f->marg_wire.size();
    out->n_meas = f->n_meas();
    out->n_slots = (int)f->slots.size();
    out->n_ops = f->clifford ? (int)f->cops.size() : (int)f->nops.size();
    out->n_moments = f->n_moments();
    out->n_zstrings = (int)f->zwires.size();
    return CCS_OK;
  });
}

int ccs_plan_cuts(ccs_ctx c, ccs_plan p, int problem, ccs_cut* out, int cap) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!p || problem < 0 || problem >= (int)p->problems.size()) return fail(c, CCS_ERR_INVALID_ARG, "bad problem");
    const auto& cuts = p->problems[problem].cuts;
    if (cap < (int)cuts.size()) return fail(c, CCS_ERR_INVALID_ARG, "buffer too small");
    for (size_t i = 0; i < cuts.size(); ++i) out[i] = cuts[i];
    return (int)cuts.size();
  });
}

int ccs_fragment_wires(ccs_ctx c, ccs_plan p, int problem, int fragment, uint32_t* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    int g;
    const Frag* f = p ? find_frag(p, problem, fragment, &g) : nullptr;
    if (!f || !out) return fail(c, CCS_ERR_INVALID_ARG, "bad fragment");
    for (int i = 0; i < f->n(); ++i) { out[2 * i] = f->wires[i].first; out[2 * i + 1] = f->wires[i].second; }
    return CCS_OK;
  });
}

static int locate(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, const FragDev** fd) {
  if (!c || !r) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
  int g;
  const Frag* f = find_frag(r->plan, problem, fragment, &g);
  if (!f) return fail(c, CCS_ERR_INVALID_ARG, "bad fragment");
  if (variant < -1 || variant >= f->n_variants()) return fail(c, CCS_ERR_INVALID_ARG, "bad variant");
  *fd = &r->plan->fdev[g];
  cudaSetDevice(c->device);
  return check_status(c, r);
}

int ccs_get_tableau(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, uint8_t* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, variant, &d);
    if (rc) return rc;
    if (!d->clifford || !r->ep.keep_tableaus || variant < 0) return fail(c, CCS_ERR_INVALID_ARG, "no tableau kept");
    const int n = d->n, W = d->W, Wh = d->Wh, ncol = 2 * n + 3;
    std::vector<unsigned long long> h((size_t)ncol * W);
    cudaError_t e = cudaMemcpy(h.data(), r->dr.tabs + d->tab_off + (long long)variant * ncol * W,
                               h.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy tableau");
    auto bit = [&](int col, int row) -> uint8_t {
      const int word = row < n ? row / 64 : Wh + (row - n) / 64;
      const int b = row < n ? row % 64 : (row - n) % 64;
      return (uint8_t)((h[(size_t)col * W + word] >> b) & 1ull);
    };
    for (int row = 0; row < 2 * n; ++row) {
      uint8_t* o = out + (size_t)row * (2 * n + 1);
      for (int j = 0; j < n; ++j) { o[j] = bit(j, row); o[n + j] = bit(n + 1 + j, row); }
      o[2 * n] = bit(2 * (n + 1), row);
    }
    return CCS_OK;
  });
}

int ccs_get_outcome_space(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, uint64_t* off,
                          uint64_t* basis, int* rank) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, variant, &d);
    if (rc) return rc;
    if (!d->clifford || variant < 0) return fail(c, CCS_ERR_INVALID_ARG, "not a Clifford variant");
    SpaceRec s;
    cudaError_t e = cudaMemcpy(&s, r->dr.spaces + d->space_off + variant, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy space");
    if (off) *off = s.off;
    if (rank) *rank = s.rank;
    if (basis)
      for (int i = 0; i < s.rank; ++i) basis[i] = s.basis[i];
    return CCS_OK;
  });
}

int ccs_get_counts(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, uint32_t* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, variant, &d);
    if (rc) return rc;
    if (!d->clifford || r->ep.mode != CCS_SAMPLED || variant < 0) return fail(c, CCS_ERR_INVALID_ARG, "no counts");
    if (d->role == 1 && !r->ep.keep_tableaus) return fail(c, CCS_ERR_INVALID_ARG, "hub counts are kept only with keep_tableaus");
    cudaError_t e = cudaMemcpy(out, r->dr.counts + d->counts_off + ((long long)variant << d->nA),
                               sizeof(uint32_t) << d->nA, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CCS_OK : cuda_fail(c, e, "copy counts");
  });
}

int ccs_get_dist(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, float* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, variant, &d);
    if (rc) return rc;
    const bool have = !d->clifford || r->ep.mode == CCS_EXACT || (r->ep.mode == CCS_STITCH && d->role != 1);
    if (!have || variant < 0) return fail(c, CCS_ERR_INVALID_ARG, "no distribution");
    cudaError_t e = cudaMemcpy(out, r->dr.dist + d->dist_off + ((long long)variant << d->nA),
                               sizeof(float) << d->nA, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CCS_OK : cuda_fail(c, e, "copy dist");
  });
}

int ccs_get_zvals(ccs_ctx c, ccs_res r, int problem, int fragment, int variant, float* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, variant, &d);
    if (rc) return rc;
    if (variant < 0) return fail(c, CCS_ERR_INVALID_ARG, "no variant");
    const long long cnt = (long long)d->nz << d->qout;
    if (cnt == 0) return CCS_OK;
    cudaError_t e = cudaMemcpy(out, r->dr.zval + d->zval_off + (long long)variant * cnt, cnt * sizeof(float),
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CCS_OK : cuda_fail(c, e, "copy Z values");
  });
}

int ccs_get_operand(ccs_ctx c, ccs_res r, int problem, int fragment, float* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, -1, &d);
    if (rc) return rc;
    if (d->role == 0) return fail(c, CCS_ERR_INVALID_ARG, "not part of a star contraction");
    const long long cnt = (1ll << d->m) << (2 * d->n_slots);
    if (d->role != 1) {
      cudaError_t e = cudaMemcpy(out, r->dr.TQ + d->T_off, cnt * sizeof(float), cudaMemcpyDeviceToHost);
      return e == cudaSuccess ? CCS_OK : cuda_fail(c, e, "copy operand");
    }
    // the hub's Q is stored transposed on the device ([d][o]); return [o][d]
    std::vector<float> t(cnt);
    cudaError_t e;
    if (r->dr.hub_i16 && d->clifford) {   // exact int16 count sums times 1/shots
      std::vector<int16_t> h(cnt);
      e = cudaMemcpy(h.data(), r->dr.TQ + d->T_off, cnt * sizeof(int16_t), cudaMemcpyDeviceToHost);
      for (long long i = 0; i < cnt; ++i) t[i] = (float)h[i] * r->dr.hub_scale;
    } else {
      e = cudaMemcpy(t.data(), r->dr.TQ + d->T_off, cnt * sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "copy operand");
    const long long M = 1ll << d->m, K = 1ll << (2 * d->n_slots);
    std::vector<uint8_t> live(K, 1);
    if (r->ep.mode == CCS_STITCH && d->clifford) {   // rows flagged zero may never have been written
      e = cudaMemcpy(live.data(), r->dr.qnz + d->qrow_off, K, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(c, e, "copy row flags");
    }
    for (long long k = 0; k < K; ++k)
      for (long long o = 0; o < M; ++o) out[o * K + k] = live[k] ? t[k * M + o] : 0.f;
    return CCS_OK;
  });
}

int ccs_ml_correct(ccs_ctx c, ccs_plan p, ccs_res r, int which) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !p || !r || r->plan != p) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (c->host_only) return fail(c, CCS_ERR_UNSUPPORTED, "host-only context cannot correct fragment models");
    if (which != CCS_ML_SAMPLED && which != CCS_ML_ALL) return fail(c, CCS_ERR_INVALID_ARG, "bad fragment selection");
    if (r->ep.mode == CCS_STITCH)
      return fail(c, CCS_ERR_INVALID_ARG, "a stitched result holds no fragment model to correct");
    cudaSetDevice(c->device);
    auto& mc = r->ml;
    const int key = which * 4 + r->ep.mode * 2 + (r->dr.hub_i16 ? 1 : 0);
    if (mc.key != key) {
      std::vector<MlFrag> recs;
      std::vector<int> leaf_idx;
      std::vector<long long> leaf_pref{0};
      std::vector<MlGroup> groups;
      long long floats = 0;
      bool i16_hub = false;
      for (int dd = 0; dd <= kMlMaxSlots; ++dd) {
        MlGroup G{dd, (int)recs.size(), 0, 0};
        for (int g = 0; g < (int)p->fdev.size(); ++g) {
          const FragDev& F = p->fdev[g];
          const bool pick = which == CCS_ML_ALL || (F.clifford && r->ep.mode == CCS_SAMPLED);
          if (!pick) continue;
          if (F.n_slots > kMlMaxSlots)
            return fail(c, CCS_ERR_UNSUPPORTED, "maximum-likelihood correction supports at most 6 cut slots per fragment");
          if (F.n_slots != dd) continue;
          const long long nb = 1ll << F.m, Dm = 1ll << dd;
          MlFrag mf{};
          mf.frag = g;
          mf.d = dd;
          mf.hub = F.role == 1 ? 1 : 0;
          mf.i16 = (mf.hub && r->dr.hub_i16 && F.clifford) ? 1 : 0;
          i16_hub = i16_hub || mf.i16;
          mf.index = (int)recs.size();
          mf.blk0 = G.blocks;
          mf.ev_off = floats;
          floats += nb * Dm;
          mf.vec_off = floats;
          floats += nb * 2 * Dm * Dm;   // complex64 eigenvectors
          mf.total = (double)(1ll << F.qin);
          recs.push_back(mf);
          G.blocks += nb;
          ++G.count;
          if (F.role == 2) {
            leaf_idx.push_back(g);
            leaf_pref.push_back(leaf_pref.back() + (nb << (2 * dd)));
          }
        }
        if (G.count) groups.push_back(G);
      }
      if (recs.empty()) {   // nothing estimated from shots: the models are exact
        mc.key = key;
        mc.n_frags = 0;
        mc.groups.clear();
        r->ml_applied = 1 + which;
        return CCS_OK;
      }
      if ((size_t)floats > mc.scratch_len) {
        mc.scratch = r->A.get<float>((size_t)floats);
        mc.scratch_len = mc.scratch ? (size_t)floats : 0;
        if (!mc.scratch) return fail(c, CCS_ERR_OOM, "correction scratch");
      }
      int* d_leaf = nullptr;
      long long* d_pref = nullptr;
      if (!upload(c, r->A, recs, &mc.d_frags) || !(mc.theta = r->A.get<double>(recs.size())) ||
          !upload(c, r->A, leaf_idx, &d_leaf) || !upload(c, r->A, leaf_pref, &d_pref))
        return fail(c, CCS_ERR_OOM, "correction records");
      mc.n_frags = (int)recs.size();
      mc.groups = groups;
      mc.leaves = FoldSet{d_leaf, d_pref, (int)leaf_idx.size(), leaf_pref.back()};
      mc.i16_hub = i16_hub;
      mc.key = key;
    }
    if (mc.n_frags == 0) {
      r->ml_applied = 1 + which;
      return CCS_OK;
    }
    cudaError_t e = launch_ml_correct(p->dp, r->dr, mc.d_frags, mc.n_frags, mc.groups.data(), (int)mc.groups.size(),
                                      mc.scratch, mc.theta, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "correction kernels");
    if (mc.i16_hub) r->dr.hub_i16 = 0;   // the corrected hub operands are FP32 now
    if (mc.leaves.nf &&
        (e = launch_operands(p->dp, r->dr, r->ep, FoldSet{nullptr, nullptr, 0, 0}, mc.leaves, c->stream)) !=
            cudaSuccess)
      return cuda_fail(c, e, "leaf operands");
    r->ml_applied = 1 + which;
    return CCS_OK;
  });
}

int ccs_get_tensor(ccs_ctx c, ccs_res r, int problem, int fragment, float* out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    const FragDev* d;
    int rc = locate(c, r, problem, fragment, -1, &d);
    if (rc) return rc;
    const long long cnt = (1ll << d->m) << (2 * d->n_slots);
    // corrected by ccs_ml_correct since the evaluation: every fragment under
    // CCS_ML_ALL, the Clifford fragments of a sampled result otherwise
    const bool corrected = r->ml_applied && (r->ml_applied == 1 + CCS_ML_ALL ||
                                             (d->clifford && r->ep.mode == CCS_SAMPLED));
    if (d->role == 1 && !corrected && d->clifford && r->ep.mode == CCS_SAMPLED && !r->ep.keep_tableaus)
      return fail(c, CCS_ERR_INVALID_ARG, "a sampled hub's tensor needs its counts (keep_tableaus)");
    if (d->role == 1 && d->clifford && r->ep.mode == CCS_STITCH)
      return fail(c, CCS_ERR_INVALID_ARG, "a stitched hub forms no per-variant distribution (see ccs_get_operand)");
    if (d->role == 1 && !corrected) {   // a hub's T is not formed on the hot path: fold it now
      const int g = (int)(d - r->plan->fdev.data());
      std::vector<int> fi{g};
      std::vector<long long> tp{0, cnt};
      Allocs tmp;
      tmp.ctx = c;
      int* dfi; long long* dtp;
      if (!upload(c, tmp, fi, &dfi) || !upload(c, tmp, tp, &dtp)) {
        tmp.release();
        return fail(c, CCS_ERR_OOM, "tensor fold buffers");
      }
      cudaError_t e2 = launch_fold(r->plan->dp, r->dr, r->ep, FoldSet{dfi, dtp, 1, cnt}, c->stream);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
      tmp.release();
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "tensor fold");
    }
    cudaError_t e = cudaMemcpy(out, r->dr.T + d->T_off, cnt * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? CCS_OK : cuda_fail(c, e, "copy tensor");
  });
}

}  // extern "C"

// --- recombination without device allocation ---------------------------------
// The scratch of the recombination (the leaves' Kronecker operand R and the
// split-K partial tiles) lives in this fixed array instead of memory the
// library allocates.  Every GPU that loads the library holds it until the
// process exits.  In host code `g_noalloc_scratch` names a host-side stand-in,
// not device memory, so its device address is looked up once per device.
namespace {
constexpr long long kNoAllocScratchFloats = 2ll << 20;   // 8 MiB of float
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];
constexpr int kMaxDevices = 64;
// device address of the array per device, looked up under the lock on the
// first call that needs it (a later cudaDeviceReset invalidates it)
std::mutex g_noalloc_mu;
float* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

extern "C" int ccs_recombine_noalloc(ccs_ctx c, ccs_plan p, ccs_res r, int precision, double* marginal_out,
                                     double* zexp_out) {
  return abi_guard([&](int code, const char* m) { return fail(c, code, m); }, [&]() -> int {
    if (!c || !p || !r || r->plan != p) return fail(c, CCS_ERR_INVALID_ARG, "bad arguments");
    if (c->host_only) return fail(c, CCS_ERR_UNSUPPORTED, "host-only context cannot recombine");
    if (precision != CCS_FP32 && precision != CCS_BF16) return fail(c, CCS_ERR_INVALID_ARG, "bad precision");
    if ((p->n_marg && !marginal_out) || (p->n_zexp && !zexp_out))
      return fail(c, CCS_ERR_INVALID_ARG, "null output buffer");
    const long long need = p->r_total + p->part_total;
    if (need > kNoAllocScratchFloats)
      return fail(c, CCS_ERR_UNSUPPORTED,
                  "recombination needs " + std::to_string(need * 4) + " bytes of scratch; the fixed scratch of "
                  "ccs_recombine_noalloc holds " + std::to_string(kNoAllocScratchFloats * 4) + " bytes");
    if (c->device < 0 || c->device >= kMaxDevices) return fail(c, CCS_ERR_UNSUPPORTED, "device index too large");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "set device");
    float* scratch = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_noalloc_mu);
      if (!g_noalloc_addr[c->device]) {   // first call on this device: resolve the array's address
        float* ptr = nullptr;
        e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress of the fixed scratch");
        g_noalloc_addr[c->device] = ptr;
      }
      scratch = g_noalloc_addr[c->device];
    }
    RecombSizes rz{p->r_total, p->part_total, p->gemm_blocks, p->n_marg, p->n_zexp,
                   p->d_direct_items, (int)p->direct_items.size(), (int)p->direct_stage_floats, p->chain,
                   p->d_r_prefix, p->d_blk_prefix, p->d_out_prefix, p->d_z_prefix, p->max_tile_smem,
                   p->pdev.data(), (int)p->pdev.size(), nullptr, 0, r->ep.mode == CCS_STITCH ? 1 : 0,
                   KRange{0, -1}, p->all_star ? 0 : 1};
    e = launch_recombine(p->dp, r->dr, precision, rz, scratch, marginal_out, zexp_out, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "recombine kernel");
    return CCS_OK;
  });
}
