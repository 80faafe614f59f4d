// C ABI of the batched GEMM library (include/bgemm.h): argument checking,
// plans (size classes, work tables, autotuning, graph capture), chained
// products, measurement entry points and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bgemm_internal.h"
#include "split.h"

namespace bg {

// ---- errors and bookkeeping ------------------------------------------------------------

static thread_local std::string g_last_error;
static thread_local int64_t g_launches = 0;

void count_launch(int n) { g_launches += n; }

static bg_status fail(bg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

static bg_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls start clean
  if (e == cudaErrorMemoryAllocation)
    return fail(BG_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorStreamCaptureUnsupported || e == cudaErrorStreamCaptureInvalidated)
    return fail(BG_ERR_CAPTURE, "%s: %s", what, cudaGetErrorString(e));
  return fail(BG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BG_CUDA(call, what)                      \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Host-side fault injection for tests: BGEMM_FAULT=launch makes every compute
// entry point fail with BG_ERR_CUDA before it launches anything.
static bool fault_injected() {
  const char* f = getenv("BGEMM_FAULT");
  return f && strcmp(f, "launch") == 0;
}

static bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Per-device state: SM count, device error word, workspace of fixed split calls.
struct DeviceCtx {
  int device = -1;
  int sms = 0;
  int* d_err = nullptr;
  SplitWorkspace ws;
  std::mutex mu;
};

static std::mutex g_ctx_mu;
static std::map<int, DeviceCtx*> g_ctx;

static bg_status get_ctx(DeviceCtx** out) {
  int dev = 0;
  BG_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  auto it = g_ctx.find(dev);
  if (it != g_ctx.end()) {
    *out = it->second;
    return BG_OK;
  }
  DeviceCtx* c = new DeviceCtx();
  c->device = dev;
  BG_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  cudaError_t e = cudaMalloc(&c->d_err, 4 * sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(error word)");
  }
  e = cudaMemset(c->d_err, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "cudaMemset(error word)");
  }
  g_ctx[dev] = c;
  *out = c;
  return BG_OK;
}

// ---- argument checks ----------------------------------------------------------------------

static bool aligned(const void* p, bg_dtype dt) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  return (a % (dt == BG_C128 ? 16u : 8u)) == 0;
}

static bg_status check_dtype(bg_dtype dt) {
  if (dt != BG_R64 && dt != BG_C128) return fail(BG_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
  return BG_OK;
}

static bg_status check_precision(const bg_precision* p, bg_precision* out) {
  bg_precision d{BG_MODE_FP64, 0, 0, 0};
  if (p) d = *p;
  if (d.mode != BG_MODE_FP64 && d.mode != BG_MODE_SPLIT_BF16)
    return fail(BG_ERR_INVALID_ARG, "unknown precision mode %d", d.mode);
  if (d.reserved != 0) return fail(BG_ERR_INVALID_ARG, "bg_precision.reserved must be 0");
  if (d.mode == BG_MODE_SPLIT_BF16) {
    if (d.slices < 1 || d.slices > kMaxSlices)
      return fail(BG_ERR_INVALID_ARG, "slices must be 1..%d, got %d", kMaxSlices, d.slices);
    if (d.beta_bits != 0 && (d.beta_bits < 2 || d.beta_bits > 8))
      return fail(BG_ERR_INVALID_ARG, "beta_bits must be 0 or 2..8, got %d", d.beta_bits);
  } else {
    d.slices = 0;
    d.beta_bits = 0;
  }
  *out = d;
  return BG_OK;
}

// herk: a Hermitian rank-k update (m == n required, the B fields unused).
static bg_status check_instance(const bg_instance& t, int64_t i, bool herk = false) {
  if (t.m < 0 || t.n < 0 || t.k < 0)
    return fail(BG_ERR_INVALID_ARG, "instance %lld: negative size", (long long)i);
  if (t.m > INT32_MAX / 2 || t.n > INT32_MAX / 2 || t.k > INT32_MAX / 2)
    return fail(BG_ERR_INVALID_ARG, "instance %lld: size too large", (long long)i);
  if (herk && t.m != t.n)
    return fail(BG_ERR_INVALID_ARG, "instance %lld: a Hermitian update needs m == n",
                (long long)i);
  if (t.lda < std::max<int64_t>(1, t.m) || (!herk && t.ldb < std::max<int64_t>(1, t.k)) ||
      t.ldc < std::max<int64_t>(1, t.m))
    return fail(BG_ERR_INVALID_ARG, "instance %lld: leading dimension below the row count",
                (long long)i);
  if (t.a_off < 0 || (!herk && t.b_off < 0) || t.c_off < 0)
    return fail(BG_ERR_INVALID_ARG, "instance %lld: negative offset", (long long)i);
  return BG_OK;
}

static Scalars make_scalars(bg_dtype dt, const void* alpha, const void* beta) {
  Scalars s;
  const double* a = static_cast<const double*>(alpha);
  const double* b = static_cast<const double*>(beta);
  s.alpha_re = a[0];
  s.alpha_im = dt == BG_C128 ? a[1] : 0.0;
  s.beta_re = b[0];
  s.beta_im = dt == BG_C128 ? b[1] : 0.0;
  s.alpha_zero = (s.alpha_re == 0.0 && s.alpha_im == 0.0);
  s.beta_zero = (s.beta_re == 0.0 && s.beta_im == 0.0);
  return s;
}

}  // namespace bg

using namespace bg;

// ---- plan object ---------------------------------------------------------------------------

struct ClassInfo {
  int64_t key_m, key_n, key_k;  // power-of-two bucket of the class
  int64_t members = 0;
  int prog = -1;
  double flops = 0.0;
  double ms = -1.0;            // timed ms of the chosen program (autotune), -1 if not timed
  std::vector<std::pair<int, double>> tried;
};

// Routes of a class that the split path computes (ClassInfo::prog, and the
// autotune cache's "prog" entry for split-mode keys): the default rule for
// the small-instance kernel, or (autotuned) the small-instance kernel for
// every member it can take, or the tile kernels only.
constexpr int PROG_SPLIT = -2;
constexpr int PROG_SPLIT_TILES = -3;
constexpr int PROG_SPLIT_SMALL = -4;
inline bool is_split_route(int prog) {
  return prog == PROG_SPLIT || prog == PROG_SPLIT_TILES || prog == PROG_SPLIT_SMALL;
}
inline int8_t split_route_of(int prog) {
  return prog == PROG_SPLIT_SMALL ? 1 : prog == PROG_SPLIT_TILES ? 2 : 0;
}
inline const char* split_route_name(int prog) {
  return prog == PROG_SPLIT_SMALL ? "split_small" : prog == PROG_SPLIT_TILES ? "split_tiles" : "split";
}

struct bg_plan {
  int device = 0;
  bg_dtype dtype = BG_R64;
  bg_precision prec{};
  uint32_t flags = 0;
  bool is_chain = false;
  int64_t count = 0;
  std::vector<bg_instance> table;
  std::vector<int> inst_class;
  std::vector<ClassInfo> classes;
  // FP64 path device tables
  int64_t* d_table = nullptr;
  int32_t* d_order = nullptr;
  WorkItem* d_items = nullptr;
  int64_t n_items = 0;
  int grid = 0;
  // chain
  int32_t walkers = 0, pool_count = 0;
  std::vector<int64_t> wn, woff, pool_n, pool_off;
  int64_t* d_wn = nullptr;
  int64_t* d_woff = nullptr;
  int64_t* d_pool_off = nullptr;
  int64_t* d_pool_n = nullptr;
  // split path
  SplitPlan* split = nullptr;
  // entropy plans (Alg. 1, Calculate Entropy): the Gram matrices' HERK plan,
  // the Gram buffer and the tridiagonal matrices of every walker
  bool is_entropy = false;
  bg_plan* gram = nullptr;
  double2* d_gram = nullptr;
  double* d_tri_d = nullptr;
  double* d_tri_e = nullptr;
  int ent_n = 0;
  // the blocked reduction of split-precision entropy plans: one grouped GEMM
  // plan per panel for the trailing update C[q:, q:] -= [V2 W2] [W2 V2]^H,
  // every walker's [V W] (tri_pstride elements apart) and the packed
  // second operand
  std::vector<bg_plan*> tri_gemm;
  int tri_nb = 0;
  int64_t tri_pstride = 0;
  double2* d_tri_p = nullptr;
  double2* d_tri_wvh = nullptr;
  double* d_tri_s = nullptr;  // Re G + Im G, walkers x K x K
  // annealing-step plans (Alg. 1): the entropy plan over the proposals, the
  // proposal buffer (walkers x 2^spins, contiguous) and the new energies
  bool is_anneal = false;
  bg_plan* ent = nullptr;
  double2* d_prop = nullptr;
  double* d_enew = nullptr;
  int32_t spins = 0;
  int64_t state_stride = 0;
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  std::vector<uintptr_t> gkey;
  cudaStream_t cap_stream = nullptr;
  int64_t workspace_bytes = 0;
  int launches_per_call = 0;
  // profiling: per call three events (start, after slot 0, after slot 1)
  // per profiled call: start, after slot 0, after slot 2, after slot 1
  std::vector<std::array<cudaEvent_t, 4>> prof_events;
  size_t prof_used = 0;
  double prof_ms[3] = {0.0, 0.0, 0.0};
  int64_t prof_calls = 0;
};

namespace {

int64_t pow2_bucket(int64_t x) {
  int64_t b = 1;
  while (b < x) b <<= 1;
  return b;
}

template <class T>
bg_status upload(T** dptr, const std::vector<T>& v, int64_t* ws_bytes) {
  const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  BG_CUDA(cudaMalloc(reinterpret_cast<void**>(dptr), bytes), "cudaMalloc(plan table)");
  if (!v.empty())
    BG_CUDA(cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice),
            "cudaMemcpy(plan table)");
  *ws_bytes += (int64_t)bytes;
  return BG_OK;
}

// Cost of a work item in per-thread DFMA units (longest-first ordering).
double item_cost(const WorkItem& w, const std::vector<int64_t>& mnk_k,
                 const std::vector<int64_t>& mnk_mn, const std::vector<int32_t>& order) {
  if (prog_is_small(w.prog)) {
    const double lanes = 32.0 * (w.r0 > 0 ? w.r0 : 1);  // threads per instance
    double c = 0;
    for (int i = 0; i < w.count; ++i) {
      const int64_t id = order[w.inst + i];
      c = std::max(c, std::ceil(mnk_mn[id] / lanes) * (double)mnk_k[id]);
    }
    return c;
  }
  int tm, tn;
  prog_tile(w.prog, &tm, &tn);
  return (double)tm * tn / kFp64Threads * (double)mnk_k[w.inst];
}

// Build the FP64 work list for instances with the given program per instance.
// `ids` are instance (or walker) ids, `sizes` their (m, n, k), `prog_of` the
// chosen program. Small-program instances are grouped in `order`, 8 to a CTA,
// or fewer (with several warps each) when there are too few of them to give
// each of the `grid` CTAs an item; items are sorted longest first.
void build_items(const std::vector<int64_t>& ids, const std::vector<std::array<int64_t, 3>>& mnk,
                 const std::vector<int>& prog_of, std::vector<WorkItem>* items,
                 std::vector<int32_t>* order, bool herk, int64_t grid) {
  items->clear();
  order->clear();
  const size_t N = mnk.size();
  std::vector<int64_t> kk(N), mn(N);
  for (size_t i = 0; i < N; ++i) {
    kk[i] = mnk[i][2];
    mn[i] = mnk[i][0] * mnk[i][1];
  }
  // small programs: group by program, sort each group by cost descending
  std::map<int, std::vector<int64_t>> small;
  for (int64_t id : ids) {
    const int p = prog_of[id];
    if (prog_is_small(p)) {
      small[p].push_back(id);
    } else {
      int tm, tn;
      prog_tile(p, &tm, &tn);
      const int64_t m = mnk[id][0], n = mnk[id][1];
      for (int64_t c0 = 0; c0 < n; c0 += tn)
        for (int64_t r0 = 0; r0 < m; r0 += tm) {
          if (herk && r0 + tm - 1 < c0) continue;  // wholly above the diagonal
          WorkItem w;
          w.inst = (int32_t)id;
          w.prog = (int16_t)p;
          w.count = 1;
          w.r0 = (int32_t)r0;
          w.c0 = (int32_t)c0;
          items->push_back(w);
        }
    }
  }
  for (auto& kv : small) {
    auto& v = kv.second;
    std::stable_sort(v.begin(), v.end(), [&](int64_t a, int64_t b) {
      return std::ceil(mn[a] / 32.0) * kk[a] > std::ceil(mn[b] / 32.0) * kk[b];
    });
    const int g = kv.first == PROG_R64_SMALL ? small_group((int64_t)v.size(), grid) : kSmallPerCta;
    for (size_t s = 0; s < v.size(); s += g) {
      WorkItem w;
      w.inst = (int32_t)order->size();
      w.prog = (int16_t)kv.first;
      w.count = (int16_t)std::min<size_t>(g, v.size() - s);
      w.r0 = kSmallPerCta / g;  // warps per instance
      w.c0 = 0;
      for (int i = 0; i < w.count; ++i) order->push_back((int32_t)v[s + i]);
      items->push_back(w);
    }
  }
  std::vector<double> cost(items->size());
  for (size_t i = 0; i < items->size(); ++i) cost[i] = item_cost((*items)[i], kk, mn, *order);
  std::vector<size_t> perm(items->size());
  for (size_t i = 0; i < perm.size(); ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  std::vector<WorkItem> sorted(items->size());
  for (size_t i = 0; i < perm.size(); ++i) sorted[i] = (*items)[perm[i]];
  items->swap(sorted);
}

// ---- autotune cache (JSON, one entry per line) --------------------------------------------

std::string gpu_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (auto& ch : s)
    if (ch == '"' || ch == '\\') ch = '_';
  return s;
}

std::string class_key(bg_dtype dt, const bg_precision& pr, const ClassInfo& c) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%s|%s%d|%lldx%lldx%lld", gpu_name().c_str(),
           dt == BG_C128 ? "c128" : "r64", pr.mode == BG_MODE_FP64 ? "fp64" : "split",
           pr.slices, (long long)c.key_m, (long long)c.key_n, (long long)c.key_k);
  return buf;
}

std::map<std::string, int> read_cache(const char* path) {
  std::map<std::string, int> out;
  if (!path) return out;
  FILE* f = fopen(path, "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char* q1 = strchr(line, '"');
    if (!q1) continue;
    char* q2 = strchr(q1 + 1, '"');
    if (!q2) continue;
    std::string key(q1 + 1, q2);
    const char* pp = strstr(q2, "\"prog\":");
    if (!pp) continue;
    int prog = -1;
    if (sscanf(pp + 7, "%d", &prog) == 1 && ((prog >= 0 && prog < PROG_COUNT) || is_split_route(prog)))
      out[key] = prog;
  }
  fclose(f);
  return out;
}

void write_cache(const char* path, const std::map<std::string, std::pair<int, double>>& entries) {
  if (!path) return;
  // merge with what is there
  std::map<std::string, std::pair<int, double>> all;
  for (auto& kv : read_cache(path)) all[kv.first] = {kv.second, -1.0};
  for (auto& kv : entries) all[kv.first] = kv.second;
  std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto& kv : all) {
    fprintf(f, "  \"%s\": {\"prog\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(), kv.second.first,
            kv.second.second, (++i < all.size()) ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

bg_status alloc_capture_stream(bg_plan* p) {
  if (!p->cap_stream)
    BG_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking), "stream create");
  return BG_OK;
}

// Times the FP64 persistent kernel on the items of one class with program
// `prog`, on scratch copies sized for those instances. Returns ms (median of 3).
bg_status time_class_fp64(bg_plan* p, int cls, int prog, cudaStream_t st, double* ms) {
  std::vector<int64_t> ids;
  std::vector<std::array<int64_t, 3>> mnk(p->count);
  std::vector<int> prog_of(p->count, -1);
  for (int64_t i = 0; i < p->count; ++i) {
    mnk[i] = {p->table[i].m, p->table[i].n, p->table[i].k};
    if (p->inst_class[i] == cls) {
      ids.push_back(i);
      prog_of[i] = prog;
    }
  }
  // Compact scratch layout: each sampled instance packed with ld = rows.
  // Sample at most ~64 MiB per operand.
  const int64_t esz = p->dtype == BG_C128 ? 16 : 8;
  std::vector<bg_instance> sub;
  std::vector<int64_t> sub_ids;
  int64_t la = 0, lb = 0, lc = 0;
  for (int64_t id : ids) {
    const bg_instance& t = p->table[id];
    const int64_t a = std::max<int64_t>(1, t.m) * std::max<int64_t>(1, t.k);
    const int64_t b = std::max<int64_t>(1, t.k) * std::max<int64_t>(1, t.n);
    const int64_t c = std::max<int64_t>(1, t.m) * std::max<int64_t>(1, t.n);
    if (!sub.empty() && (la + a) * esz > (64ll << 20)) break;
    bg_instance s{t.m, t.n, t.k, std::max<int64_t>(1, t.m), std::max<int64_t>(1, t.k),
                  std::max<int64_t>(1, t.m), la, lb, lc};
    la += a; lb += b; lc += c;
    sub.push_back(s);
  }
  if (sub.empty()) {
    *ms = 0;
    return BG_OK;
  }
  std::vector<int64_t> sids(sub.size());
  std::vector<std::array<int64_t, 3>> smnk(sub.size());
  std::vector<int> sprog(sub.size(), prog);
  for (size_t i = 0; i < sub.size(); ++i) {
    sids[i] = (int64_t)i;
    smnk[i] = {sub[i].m, sub[i].n, sub[i].k};
  }
  std::vector<WorkItem> items;
  std::vector<int32_t> order;
  build_items(sids, smnk, sprog, &items, &order, false, p->grid);
  void *A = nullptr, *B = nullptr, *C = nullptr;
  int64_t* dt = nullptr;
  int32_t* dord = nullptr;
  WorkItem* dit = nullptr;
  int64_t dummy = 0;
  std::vector<int64_t> flat(sub.size() * 9);
  for (size_t i = 0; i < sub.size(); ++i) memcpy(&flat[9 * i], &sub[i], 9 * sizeof(int64_t));
  bg_status rs = BG_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<float> times;
  do {
    if (cudaMalloc(&A, la * esz) != cudaSuccess || cudaMalloc(&B, lb * esz) != cudaSuccess ||
        cudaMalloc(&C, lc * esz) != cudaSuccess) {
      rs = fail(BG_ERR_NOMEM, "autotune scratch allocation failed");
      break;
    }
    cudaMemsetAsync(A, 0, la * esz, st);
    cudaMemsetAsync(B, 0, lb * esz, st);
    cudaMemsetAsync(C, 0, lc * esz, st);
    if ((rs = upload(&dt, flat, &dummy)) != BG_OK) break;
    if ((rs = upload(&dord, order, &dummy)) != BG_OK) break;
    if ((rs = upload(&dit, items, &dummy)) != BG_OK) break;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Scalars s;
    s.alpha_re = 1.0; s.alpha_im = 0.0; s.beta_re = 0.0; s.beta_im = 0.0;
    s.alpha_zero = 0; s.beta_zero = 1;
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, st);
      cudaError_t e = launch_fp64_table(p->dtype, dt, dord, dit, (int64_t)items.size(), A, B, C,
                                        s, p->grid, st);
      cudaEventRecord(e1, st);
      if (e != cudaSuccess) {
        rs = cuda_fail(e, "autotune launch");
        break;
      }
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) times.push_back(t);
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(A); cudaFree(B); cudaFree(C); cudaFree(dt); cudaFree(dord); cudaFree(dit);
  if (rs != BG_OK) return rs;
  std::sort(times.begin(), times.end());
  // scale the sampled time to the whole class by flops
  double sflops = 0, cflops = 0;
  for (auto& s : sub) sflops += (double)s.m * s.n * s.k;
  for (int64_t id : ids) cflops += (double)p->table[id].m * p->table[id].n * p->table[id].k;
  *ms = times.empty() ? 0.0 : times[times.size() / 2] * (sflops > 0 ? cflops / sflops : 1.0);
  return BG_OK;
}

void destroy_plan(bg_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (auto& ev : p->prof_events)
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  cudaFree(p->d_table);
  cudaFree(p->d_order);
  cudaFree(p->d_items);
  cudaFree(p->d_wn);
  cudaFree(p->d_woff);
  cudaFree(p->d_pool_off);
  cudaFree(p->d_pool_n);
  if (p->split) split_plan_destroy(p->split);
  if (p->gram) destroy_plan(p->gram);
  for (bg_plan* g : p->tri_gemm) destroy_plan(g);
  cudaFree(p->d_tri_p);
  cudaFree(p->d_tri_wvh);
  cudaFree(p->d_tri_s);
  if (p->ent) destroy_plan(p->ent);
  cudaFree(p->d_prop);
  cudaFree(p->d_enew);
  cudaFree(p->d_gram);
  cudaFree(p->d_tri_d);
  cudaFree(p->d_tri_e);
  cudaSetDevice(cur);
  delete p;
}

// Times the split path (slicer and tensor-core GEMM) on a compact zeroed sample
// of one class (at most about 64 MiB per operand), scaled to the whole class
// by flops. Returns ms (median of 3 runs after one warm-up).
bg_status time_class_split(bg_plan* p, int cls, cudaStream_t st, double* ms, int8_t route) {
  const int64_t esz = p->dtype == BG_C128 ? 16 : 8;
  const bool herk = (p->flags & BG_PLAN_HERK) != 0;
  std::vector<bg_instance> sub;
  int64_t la = 0, lb = 0, lc = 0;
  double sflops = 0, cflops = 0;
  for (int64_t i = 0; i < p->count; ++i) {
    if (p->inst_class[i] != cls) continue;
    const bg_instance& t = p->table[i];
    cflops += (double)t.m * t.n * t.k;
    const int64_t a = std::max<int64_t>(1, t.m) * std::max<int64_t>(1, t.k);
    const int64_t b = std::max<int64_t>(1, t.k) * std::max<int64_t>(1, t.n);
    const int64_t c = std::max<int64_t>(1, t.m) * std::max<int64_t>(1, t.n);
    if (!sub.empty() && (la + a) * esz > (64ll << 20)) continue;
    sub.push_back(bg_instance{t.m, t.n, t.k, std::max<int64_t>(1, t.m),
                              std::max<int64_t>(1, t.k), std::max<int64_t>(1, t.m), la, lb, lc});
    sflops += (double)t.m * t.n * t.k;
    la += a;
    lb += b;
    lc += c;
  }
  *ms = 0;
  if (sub.empty() || sflops == 0) return BG_OK;
  DeviceCtx* ctx;
  bg_status rs = get_ctx(&ctx);
  if (rs != BG_OK) return rs;
  SplitPlan* sp = nullptr;
  const std::vector<int8_t> routes(sub.size(), route);
  rs = split_plan_create(&sp, p->dtype, p->prec, sub, nullptr, ctx->sms, false, st,
                         &g_last_error, herk, (p->flags & BG_PLAN_SPLIT_TILES) == 0, &routes);
  if (rs != BG_OK) return rs;
  void *A = nullptr, *B = nullptr, *C = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<float> times;
  do {
    if (cudaMalloc(&A, la * esz) != cudaSuccess || cudaMalloc(&B, lb * esz) != cudaSuccess ||
        cudaMalloc(&C, lc * esz) != cudaSuccess) {
      rs = fail(BG_ERR_NOMEM, "autotune scratch allocation failed");
      break;
    }
    cudaMemsetAsync(A, 0, la * esz, st);
    cudaMemsetAsync(B, 0, lb * esz, st);
    cudaMemsetAsync(C, 0, lc * esz, st);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Scalars s;
    s.alpha_re = 1.0; s.alpha_im = 0.0; s.beta_re = 0.0; s.beta_im = 0.0;
    s.alpha_zero = 0; s.beta_zero = 1;
    for (int r = 0; r < 4 && rs == BG_OK; ++r) {
      cudaEventRecord(e0, st);
      rs = split_plan_run(sp, A, B, C, s, ctx->d_err, st, &g_last_error);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float tm = 0;
      cudaEventElapsedTime(&tm, e0, e1);
      if (r > 0) times.push_back(tm);
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(A); cudaFree(B); cudaFree(C);
  split_plan_destroy(sp);
  if (rs != BG_OK) return rs;
  std::sort(times.begin(), times.end());
  *ms = times.empty() ? 0.0 : times[times.size() / 2] * cflops / sflops;
  return BG_OK;
}

// Chooses one FP64 program per class (default or autotuned) and builds the
// device work list of the FP64 path.
//
// Split mode: without BG_PLAN_AUTOTUNE every class goes to the split path and
// no FP64 work is built. With it, each class's split time is measured beside
// its best FP64 program's, and the class is computed by whichever is faster
// (the FP64 path is never less accurate than the split modes); the choice is
// cached like the FP64 programs (key with the split mode and slice count).
bg_status build_fp64_schedule(bg_plan* p, const char* cache_path, cudaStream_t st) {
  const bool tune = (p->flags & BG_PLAN_AUTOTUNE) != 0;
  const bool split = p->prec.mode != BG_MODE_FP64;
  const bool use_cache = (p->flags & BG_PLAN_USE_CACHE) != 0 && cache_path;
  std::map<std::string, int> cache;
  if (use_cache) cache = read_cache(cache_path);
  std::map<std::string, std::pair<int, double>> new_entries;
  for (size_t c = 0; c < p->classes.size(); ++c) {
    ClassInfo& ci = p->classes[c];
    // candidate programs: those that fit every member
    std::vector<int> cand;
    const int progs_r[] = {PROG_R64_SMALL, PROG_R64_TILE, PROG_R64_DMMA};
    const int progs_c[] = {PROG_C128_SMALL, PROG_C128_TILE};
    const int* pl = p->dtype == BG_C128 ? progs_c : progs_r;
    const int np = p->dtype == BG_C128 ? 2 : 3;
    for (int q = 0; q < np; ++q) {
      bool ok = true;
      for (int64_t i = 0; i < p->count && ok; ++i)
        if (p->inst_class[i] == (int)c) ok = prog_fits(pl[q], p->dtype, p->table[i].m, p->table[i].n);
      if (ok) cand.push_back(pl[q]);
    }
    // default: small if it fits, else the DFMA tile
    int def = cand.empty() ? -1 : cand[0];
    if (p->dtype == BG_R64 && def == PROG_R64_DMMA) def = PROG_R64_TILE;
    for (int q : cand)
      if (q == PROG_R64_SMALL || q == PROG_C128_SMALL) def = q;
    if (std::find(cand.begin(), cand.end(), def) == cand.end() && !cand.empty()) def = cand[0];
    ci.prog = def;
    if (split && !tune) {
      ci.prog = PROG_SPLIT;
      continue;
    }
    const std::string key = class_key(p->dtype, p->prec, ci);
    if (use_cache && cache.count(key) &&
        (std::find(cand.begin(), cand.end(), cache[key]) != cand.end() ||
         (split && is_split_route(cache[key])))) {
      ci.prog = cache[key];
      continue;
    }
    if (tune && (cand.size() > 1 || split)) {
      double best = 1e300;
      for (int q : cand) {
        double ms = 0;
        bg_status s = time_class_fp64(p, (int)c, q, st, &ms);
        if (s != BG_OK) return s;
        ci.tried.push_back({q, ms});
        if (ms < best) {
          best = ms;
          ci.prog = q;
          ci.ms = ms;
        }
      }
      if (split) {
        // classes the small-instance kernel can take (real, m, n, k <= 64)
        // are timed on it and on the tile kernels; others on the split path
        const int beta = p->prec.beta_bits ? p->prec.beta_bits : split_default_beta(p->prec.slices);
        const bool two = p->dtype == BG_R64 && !(p->flags & BG_PLAN_HERK) &&
                         !(p->flags & BG_PLAN_SPLIT_TILES) &&
                         splitk::split_small_supported(p->prec.slices, beta) && ci.key_m <= 64 &&
                         ci.key_n <= 64 && ci.key_k <= 64;
        const int routes[2] = {two ? PROG_SPLIT_SMALL : PROG_SPLIT, PROG_SPLIT_TILES};
        for (int r = 0; r < (two ? 2 : 1); ++r) {
          double ms = 0;
          bg_status s = time_class_split(p, (int)c, st, &ms, split_route_of(routes[r]));
          if (s != BG_OK) return s;
          ci.tried.push_back({routes[r], ms});
          if (ms <= best) {
            best = ms;
            ci.prog = routes[r];
            ci.ms = ms;
          }
        }
      }
      new_entries[key] = {ci.prog, ci.ms};
    }
  }
  if (use_cache && !new_entries.empty()) write_cache(cache_path, new_entries);

  std::vector<int64_t> ids(p->count);
  std::vector<std::array<int64_t, 3>> mnk(p->count);
  std::vector<int> prog_of(p->count);
  for (int64_t i = 0; i < p->count; ++i) {
    ids[i] = i;
    mnk[i] = {p->table[i].m, p->table[i].n, p->table[i].k};
    // empty outputs need no work; alpha == 0 is handled at run time by the programs
    prog_of[i] = p->classes[p->inst_class[i]].prog;
  }
  std::vector<int64_t> live;
  for (int64_t i = 0; i < p->count; ++i)
    if (p->table[i].m > 0 && p->table[i].n > 0 && !is_split_route(prog_of[i])) live.push_back(i);
  std::vector<WorkItem> items;
  std::vector<int32_t> order;
  build_items(live, mnk, prog_of, &items, &order, (p->flags & BG_PLAN_HERK) != 0, p->grid);
  p->n_items = (int64_t)items.size();
  bg_status s;
  if ((s = upload(&p->d_order, order, &p->workspace_bytes)) != BG_OK) return s;
  if ((s = upload(&p->d_items, items, &p->workspace_bytes)) != BG_OK) return s;
  return BG_OK;
}

void assign_classes(bg_plan* p) {
  std::map<std::array<int64_t, 3>, int> idx;
  p->inst_class.assign(p->count, 0);
  p->classes.clear();
  for (int64_t i = 0; i < p->count; ++i) {
    const bg_instance& t = p->table[i];
    std::array<int64_t, 3> key = {pow2_bucket(t.m), pow2_bucket(t.n), pow2_bucket(t.k)};
    auto it = idx.find(key);
    int c;
    if (it == idx.end()) {
      c = (int)p->classes.size();
      idx[key] = c;
      ClassInfo ci;
      ci.key_m = key[0];
      ci.key_n = key[1];
      ci.key_k = key[2];
      p->classes.push_back(ci);
    } else {
      c = it->second;
    }
    p->inst_class[i] = c;
    p->classes[c].members++;
    p->classes[c].flops += (p->dtype == BG_C128 ? 8.0 : 2.0) * (double)t.m * t.n * t.k;
  }
}

}  // namespace

// ---- entry points ------------------------------------------------------------------------

extern "C" {

// Checks shared by the two fixed-size entry points. Sets *nothing_to_do for an
// empty batch (m, n or batch zero), which both treat as a no-op.
static bg_status check_fixed(bg_dtype dtype, int64_t m, int64_t n, int64_t k, const void* alpha,
                             const void* A, int64_t lda, int64_t strideA, const void* B,
                             int64_t ldb, int64_t strideB, const void* beta, void* C, int64_t ldc,
                             int64_t strideC, int64_t batch, const bg_precision* precision,
                             bg_precision* pr, Scalars* sc, bool* nothing_to_do) {
  *nothing_to_do = false;
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  if ((s = check_precision(precision, pr)) != BG_OK) return s;
  if (m < 0 || n < 0 || k < 0 || batch < 0)
    return fail(BG_ERR_INVALID_ARG, "negative size (m=%lld n=%lld k=%lld batch=%lld)",
                (long long)m, (long long)n, (long long)k, (long long)batch);
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2)
    return fail(BG_ERR_INVALID_ARG, "size too large");
  if (lda < std::max<int64_t>(1, m) || ldb < std::max<int64_t>(1, k) ||
      ldc < std::max<int64_t>(1, m))
    return fail(BG_ERR_INVALID_ARG, "leading dimension below the row count");
  if (strideA < 0 || strideB < 0 || strideC < 0)
    return fail(BG_ERR_INVALID_ARG, "negative stride");
  if (batch == 0 || m == 0 || n == 0) {
    *nothing_to_do = true;
    return BG_OK;
  }
  if (!alpha || !beta) return fail(BG_ERR_INVALID_ARG, "alpha and beta must be host pointers");
  *sc = make_scalars(dtype, alpha, beta);
  if (!C || (!sc->alpha_zero && k > 0 && (!A || !B)))
    return fail(BG_ERR_INVALID_ARG, "null matrix pointer");
  if (!aligned(C, dtype) || (A && !aligned(A, dtype)) || (B && !aligned(B, dtype)))
    return fail(BG_ERR_INVALID_ARG, "matrix pointer not %d-byte aligned", dtype == BG_C128 ? 16 : 8);
  if (strideC > 0 && strideC < ldc * (n - 1) + m && batch > 1)
    return fail(BG_ERR_INVALID_ARG, "strideC makes C instances overlap");
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch fault (BGEMM_FAULT=launch)");
  return BG_OK;
}

bg_status batched_gemm_fixed(bg_dtype dtype, int64_t m, int64_t n, int64_t k, const void* alpha,
                             const void* A, int64_t lda, int64_t strideA, const void* B,
                             int64_t ldb, int64_t strideB, const void* beta, void* C, int64_t ldc,
                             int64_t strideC, int64_t batch, const bg_precision* precision,
                             bg_stream_t stream) {
  bg_precision pr;
  Scalars sc;
  bool empty = false;
  bg_status s = check_fixed(dtype, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc,
                            strideC, batch, precision, &pr, &sc, &empty);
  if (s != BG_OK || empty) return s;
  DeviceCtx* ctx;
  if ((s = get_ctx(&ctx)) != BG_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pr.mode == BG_MODE_FP64) {
    const int prog = default_prog(dtype, m, n, k);
    cudaError_t e = launch_fp64_fixed(dtype, prog, m, n, k, sc, A, lda, strideA, B, ldb, strideB,
                                      C, ldc, strideC, batch, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "FP64 batched kernel launch");
    return BG_OK;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  return split_fixed(dtype, pr, m, n, k, sc, A, lda, strideA, B, ldb, strideB, C, ldc, strideC,
                     batch, &ctx->ws, ctx->sms, ctx->d_err, stream_capturing(st), st,
                     &g_last_error);
}

bg_status batched_gemm_fixed_static(bg_dtype dtype, int64_t m, int64_t n, int64_t k,
                                    const void* alpha, const void* A, int64_t lda,
                                    int64_t strideA, const void* B, int64_t ldb, int64_t strideB,
                                    const void* beta, void* C, int64_t ldc, int64_t strideC,
                                    int64_t batch, const bg_precision* precision,
                                    bg_stream_t stream) {
  bg_precision pr;
  Scalars sc;
  bool empty = false;
  bg_status s = check_fixed(dtype, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc,
                            strideC, batch, precision, &pr, &sc, &empty);
  if (s != BG_OK) return s;
  if (pr.mode != BG_MODE_SPLIT_BF16)
    return fail(BG_ERR_INVALID_ARG,
                "batched_gemm_fixed_static runs the split mode only (precision.mode must be "
                "BG_MODE_SPLIT_BF16)");
  if (empty) return BG_OK;
  // The call uploads its work tables from host vectors freed on return: a
  // captured copy would read freed memory when the graph replays.
  if (stream_capturing(reinterpret_cast<cudaStream_t>(stream)))
    return fail(BG_ERR_CAPTURE,
                "batched_gemm_fixed_static uploads host tables on every call; the stream is "
                "being captured");
  int dev = 0, sms = 0;
  BG_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  BG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  void* scratch = nullptr;
  size_t bytes = 0;
  if ((s = static_scratch(&scratch, &bytes, &g_last_error)) != BG_OK) return s;
  return split_fixed_in_scratch(dtype, pr, m, n, k, sc, A, lda, strideA, B, ldb, strideB, C, ldc,
                                strideC, batch, scratch, bytes, sms,
                                reinterpret_cast<cudaStream_t>(stream), &g_last_error);
}

bg_status batched_gemm_plan(bg_plan** out, bg_dtype dtype, int64_t count,
                            const bg_instance* host_table, const bg_precision* precision,
                            uint32_t flags, const char* cache_path, bg_stream_t stream) {
  if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  bg_precision pr;
  if ((s = check_precision(precision, &pr)) != BG_OK) return s;
  if (count < 0) return fail(BG_ERR_INVALID_ARG, "negative count");
  if (count > INT32_MAX / 2) return fail(BG_ERR_INVALID_ARG, "count too large");
  if (count > 0 && !host_table) return fail(BG_ERR_INVALID_ARG, "host_table is NULL");
  if (flags & ~63u) return fail(BG_ERR_INVALID_ARG, "unknown plan flags 0x%x", flags);
  const bool herk = (flags & BG_PLAN_HERK) != 0;
  for (int64_t i = 0; i < count; ++i)
    if ((s = check_instance(host_table[i], i, herk)) != BG_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (stream_capturing(st))
    return fail(BG_ERR_CAPTURE, "batched_gemm_plan allocates; the stream is being captured");
  DeviceCtx* ctx;
  if ((s = get_ctx(&ctx)) != BG_OK) return s;
  bg_plan* p = new bg_plan();
  p->device = ctx->device;
  p->dtype = dtype;
  p->prec = pr;
  p->flags = flags;
  p->count = count;
  p->table.assign(host_table, host_table + count);
  p->grid = ctx->sms * fp64_blocks_per_sm(dtype);
  assign_classes(p);
  std::vector<int64_t> flat(count * 9);
  for (int64_t i = 0; i < count; ++i) memcpy(&flat[9 * i], &p->table[i], 9 * sizeof(int64_t));
  if ((s = upload(&p->d_table, flat, &p->workspace_bytes)) != BG_OK) {
    destroy_plan(p);
    return s;
  }
  if (pr.mode == BG_MODE_FP64) {
    if ((s = build_fp64_schedule(p, cache_path, st)) != BG_OK) {
      destroy_plan(p);
      return s;
    }
    p->launches_per_call = p->n_items > 0 ? 1 : 0;
  } else {
    // each class to the split path, or (autotuned) to the FP64 path where that is faster
    if ((s = build_fp64_schedule(p, cache_path, st)) != BG_OK) {
      destroy_plan(p);
      return s;
    }
    std::vector<bg_instance> sub;
    std::vector<int8_t> routes;
    for (int64_t i = 0; i < count; ++i) {
      const int prog = p->classes[p->inst_class[i]].prog;
      if (is_split_route(prog)) {
        sub.push_back(p->table[i]);
        routes.push_back(split_route_of(prog));
      }
    }
    if (!sub.empty()) {
      s = split_plan_create(&p->split, dtype, pr, sub, nullptr, ctx->sms, false, st,
                            &g_last_error, herk, (flags & BG_PLAN_SPLIT_TILES) == 0, &routes);
      if (s != BG_OK) {
        destroy_plan(p);
        return s;
      }
      p->workspace_bytes += split_plan_workspace(p->split);
    }
    p->launches_per_call =
        (p->split ? split_plan_launches(p->split) : 0) + (p->n_items > 0 ? 1 : 0);
  }
  *out = p;
  return BG_OK;
}

static bg_status run_grouped_direct(bg_plan* p, const void* A, const void* B, void* C,
                                    const Scalars& sc, cudaStream_t st) {
  cudaEvent_t* ev = nullptr;
  if (p->flags & BG_PLAN_PROFILE) {
    if (p->prof_used == p->prof_events.size()) {
      std::array<cudaEvent_t, 4> t{};
      for (auto& e : t) BG_CUDA(cudaEventCreate(&e), "profiling event");
      p->prof_events.push_back(t);
    }
    ev = p->prof_events[p->prof_used++].data();
    BG_CUDA(cudaEventRecord(ev[0], st), "profiling event record");
  }
  if (p->prec.mode == BG_MODE_FP64) {
    cudaError_t e = launch_fp64_table(p->dtype, p->d_table, p->d_order, p->d_items, p->n_items, A,
                                      B, C, sc, p->grid, st, (p->flags & BG_PLAN_HERK) != 0);
    if (e != cudaSuccess) return cuda_fail(e, "grouped FP64 launch");
    if (ev)
      for (int i = 1; i < 4; ++i) BG_CUDA(cudaEventRecord(ev[i], st), "profiling event record");
    return BG_OK;
  }
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  if (p->split) {
    s = split_plan_run(p->split, A, B, C, sc, ctx->d_err, st, &g_last_error,
                       ev ? ev + 1 : nullptr);
    if (s != BG_OK) return s;
  } else if (ev) {
    for (int i = 1; i < 4; ++i) BG_CUDA(cudaEventRecord(ev[i], st), "profiling event record");
  }
  if (p->n_items > 0) {
    // classes the autotuner gave to the FP64 path (timed with the GEMM slot)
    cudaError_t e = launch_fp64_table(p->dtype, p->d_table, p->d_order, p->d_items, p->n_items, A,
                                      B, C, sc, p->grid, st, (p->flags & BG_PLAN_HERK) != 0);
    if (e != cudaSuccess) return cuda_fail(e, "grouped FP64 launch");
    if (ev) BG_CUDA(cudaEventRecord(ev[3], st), "profiling event record");
  }
  return BG_OK;
}

bg_status batched_gemm_grouped(const bg_plan* plan, const void* A_base, const void* B_base,
                               void* C_base, const void* alpha, const void* beta,
                               bg_stream_t stream) {
  if (!plan) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
  if (plan->is_chain) return fail(BG_ERR_INVALID_ARG, "chain plans run through chain_step");
  if (plan->is_entropy || plan->is_anneal)
    return fail(BG_ERR_INVALID_ARG, "entropy and annealing plans have their own run calls");
  if (plan->count == 0) return BG_OK;
  if (!alpha || !beta) return fail(BG_ERR_INVALID_ARG, "alpha and beta must be host pointers");
  const Scalars sc = make_scalars(plan->dtype, alpha, beta);
  const bool herk = (plan->flags & BG_PLAN_HERK) != 0;
  if (herk && (sc.alpha_im != 0.0 || sc.beta_im != 0.0))
    return fail(BG_ERR_INVALID_ARG, "a Hermitian update takes real alpha and beta");
  if (!C_base || (!sc.alpha_zero && (!A_base || (!herk && !B_base))))
    return fail(BG_ERR_INVALID_ARG, "null base pointer");
  if (!aligned(C_base, plan->dtype) || (A_base && !aligned(A_base, plan->dtype)) ||
      (B_base && !aligned(B_base, plan->dtype)))
    return fail(BG_ERR_INVALID_ARG, "base pointer misaligned");
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch fault (BGEMM_FAULT=launch)");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != plan->device) return fail(BG_ERR_INVALID_ARG, "plan belongs to another device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bg_plan* p = const_cast<bg_plan*>(plan);
  const bool want_graph = (p->flags & BG_PLAN_CAPTURE_GRAPH) != 0 &&
                          (p->flags & BG_PLAN_PROFILE) == 0 && !stream_capturing(st);
  if (!want_graph) return run_grouped_direct(p, A_base, B_base, C_base, sc, st);
  uint64_t ab[4];
  memcpy(&ab[0], &sc.alpha_re, 8);
  memcpy(&ab[1], &sc.alpha_im, 8);
  memcpy(&ab[2], &sc.beta_re, 8);
  memcpy(&ab[3], &sc.beta_im, 8);
  std::vector<uintptr_t> key = {reinterpret_cast<uintptr_t>(A_base),
                                reinterpret_cast<uintptr_t>(B_base),
                                reinterpret_cast<uintptr_t>(C_base), (uintptr_t)ab[0],
                                (uintptr_t)ab[1], (uintptr_t)ab[2], (uintptr_t)ab[3]};
  if (!p->gexec || p->gkey != key) {
    bg_status s = alloc_capture_stream(p);
    if (s != BG_OK) return s;
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    BG_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    const int64_t before = g_launches;
    s = run_grouped_direct(p, A_base, B_base, C_base, sc, p->cap_stream);
    g_launches = before;  // captured, not launched
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (s != BG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->gkey = key;
  }
  BG_CUDA(cudaGraphLaunch(p->gexec, st), "graph launch");
  count_launch(p->launches_per_call);
  return BG_OK;
}

bg_status chain_plan(bg_plan** out, bg_dtype dtype, int32_t walkers, const int64_t* walker_n,
                     const int64_t* state_off, int32_t pool_count, const int64_t* pool_n,
                     const int64_t* pool_off, const bg_precision* precision, uint32_t flags,
                     bg_stream_t stream) {
  if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  bg_precision pr;
  if ((s = check_precision(precision, &pr)) != BG_OK) return s;
  if (walkers < 0 || pool_count < 0) return fail(BG_ERR_INVALID_ARG, "negative count");
  if (walkers > 0 && (!walker_n || !state_off))
    return fail(BG_ERR_INVALID_ARG, "walker arrays are NULL");
  if (pool_count > 0 && (!pool_n || !pool_off))
    return fail(BG_ERR_INVALID_ARG, "pool arrays are NULL");
  if (flags & ~15u) return fail(BG_ERR_INVALID_ARG, "unknown plan flags 0x%x", flags);
  for (int32_t w = 0; w < walkers; ++w) {
    if (walker_n[w] < 0 || walker_n[w] > 65536 || state_off[w] < 0)
      return fail(BG_ERR_INVALID_ARG, "walker %d: bad size or offset", w);
    bool found = false;
    for (int32_t j = 0; j < pool_count && !found; ++j) found = pool_n[j] == walker_n[w];
    if (!found && walker_n[w] > 0)
      return fail(BG_ERR_INVALID_ARG, "walker %d: no pool matrix of size %lld", w,
                  (long long)walker_n[w]);
  }
  for (int32_t j = 0; j < pool_count; ++j)
    if (pool_n[j] < 0 || pool_off[j] < 0)
      return fail(BG_ERR_INVALID_ARG, "pool entry %d: bad size or offset", j);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (stream_capturing(st))
    return fail(BG_ERR_CAPTURE, "chain_plan allocates; the stream is being captured");
  DeviceCtx* ctx;
  if ((s = get_ctx(&ctx)) != BG_OK) return s;
  bg_plan* p = new bg_plan();
  p->device = ctx->device;
  p->dtype = dtype;
  p->prec = pr;
  p->flags = flags;
  p->is_chain = true;
  p->walkers = walkers;
  p->pool_count = pool_count;
  p->wn.assign(walker_n, walker_n + walkers);
  p->woff.assign(state_off, state_off + walkers);
  p->pool_n.assign(pool_n, pool_n + pool_count);
  p->pool_off.assign(pool_off, pool_off + pool_count);
  p->count = walkers;
  p->grid = ctx->sms * fp64_blocks_per_sm(dtype);
  // walkers as instances n x n x n (offsets unused by the FP64 chain source)
  for (int32_t w = 0; w < walkers; ++w) {
    const int64_t n = walker_n[w];
    bg_instance t{n, n, n, std::max<int64_t>(1, n), std::max<int64_t>(1, n),
                  std::max<int64_t>(1, n), 0, state_off[w], state_off[w]};
    p->table.push_back(t);
  }
  assign_classes(p);
  if ((s = upload(&p->d_wn, p->wn, &p->workspace_bytes)) != BG_OK ||
      (s = upload(&p->d_woff, p->woff, &p->workspace_bytes)) != BG_OK ||
      (s = upload(&p->d_pool_off, p->pool_off, &p->workspace_bytes)) != BG_OK ||
      (s = upload(&p->d_pool_n, p->pool_n, &p->workspace_bytes)) != BG_OK) {
    destroy_plan(p);
    return s;
  }
  if (pr.mode == BG_MODE_FP64) {
    if ((s = build_fp64_schedule(p, nullptr, st)) != BG_OK) {
      destroy_plan(p);
      return s;
    }
    p->launches_per_call = p->n_items > 0 ? 1 : 0;  // per step
  } else {
    s = split_chain_create(&p->split, dtype, pr, p->wn, p->woff, p->pool_n, p->pool_off,
                           ctx->sms, st, &g_last_error);
    if (s != BG_OK) {
      destroy_plan(p);
      return s;
    }
    p->workspace_bytes += split_plan_workspace(p->split);
    p->launches_per_call = split_plan_launches(p->split);
  }
  *out = p;
  return BG_OK;
}

static bg_status run_chain_direct(bg_plan* p, const void* U, const int32_t* idx, void* ping,
                                  void* pong, int32_t steps, cudaStream_t st) {
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  if (p->prec.mode != BG_MODE_FP64) {
    s = split_chain_prepare_pool(p->split, U, ctx->d_err, st, &g_last_error);
    if (s != BG_OK) return s;
  }
  for (int32_t t = 0; t < steps; ++t) {
    const void* cin = (t % 2 == 0) ? ping : pong;
    void* cout = (t % 2 == 0) ? pong : ping;
    const int32_t* row = idx + (int64_t)t * p->walkers;
    if (p->prec.mode == BG_MODE_FP64) {
      cudaError_t e = launch_fp64_chain(p->dtype, p->d_wn, p->d_woff, p->d_pool_off, p->d_pool_n,
                                        p->pool_count, p->d_order,
                                        row, p->d_items, p->n_items, U, cin, cout, p->grid, st);
      if (e != cudaSuccess) return cuda_fail(e, "chain step launch");
    } else {
      s = split_chain_step(p->split, U, row, cin, cout, ctx->d_err, st, &g_last_error);
      if (s != BG_OK) return s;
    }
  }
  return BG_OK;
}

bg_status chain_step(const bg_plan* plan, const void* U_pool, const int32_t* U_index,
                     void* C_ping, void* C_pong, int32_t steps, bg_stream_t stream) {
  if (!plan) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->is_chain) return fail(BG_ERR_INVALID_ARG, "not a chain plan (use chain_plan)");
  if (steps < 0) return fail(BG_ERR_INVALID_ARG, "negative steps");
  if (steps == 0 || plan->walkers == 0) return BG_OK;
  if (!U_pool || !U_index || !C_ping || !C_pong)
    return fail(BG_ERR_INVALID_ARG, "null pointer");
  if (C_ping == C_pong) return fail(BG_ERR_INVALID_ARG, "C_ping and C_pong must differ");
  if (!aligned(U_pool, plan->dtype) || !aligned(C_ping, plan->dtype) ||
      !aligned(C_pong, plan->dtype) || (reinterpret_cast<uintptr_t>(U_index) % 4) != 0)
    return fail(BG_ERR_INVALID_ARG, "pointer misaligned");
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch fault (BGEMM_FAULT=launch)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bg_plan* p = const_cast<bg_plan*>(plan);
  const bool want_graph = (p->flags & BG_PLAN_CAPTURE_GRAPH) != 0 && !stream_capturing(st);
  if (!want_graph) return run_chain_direct(p, U_pool, U_index, C_ping, C_pong, steps, st);
  std::vector<uintptr_t> key = {reinterpret_cast<uintptr_t>(U_pool),
                                reinterpret_cast<uintptr_t>(U_index),
                                reinterpret_cast<uintptr_t>(C_ping),
                                reinterpret_cast<uintptr_t>(C_pong), (uintptr_t)steps};
  if (!p->gexec || p->gkey != key) {
    bg_status s = alloc_capture_stream(p);
    if (s != BG_OK) return s;
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    BG_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    const int64_t before = g_launches;
    s = run_chain_direct(p, U_pool, U_index, C_ping, C_pong, steps, p->cap_stream);
    const int64_t captured = g_launches - before;
    g_launches = before;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (s != BG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    p->gkey = key;
    p->launches_per_call = (int)std::max<int64_t>(0, captured / std::max<int32_t>(1, steps));
  }
  BG_CUDA(cudaGraphLaunch(p->gexec, st), "graph launch");
  count_launch(p->launches_per_call * steps);
  return BG_OK;
}

void bg_plan_destroy(bg_plan* plan) { destroy_plan(plan); }

bg_status bg_plan_kernel_times(const bg_plan* plan, int32_t reset, double* total_ms,
                               int64_t* calls) {
  if (!plan || !total_ms || !calls) return fail(BG_ERR_INVALID_ARG, "null pointer");
  bg_plan* p = const_cast<bg_plan*>(plan);
  for (size_t i = 0; i < p->prof_used; ++i) {
    cudaEvent_t* ev = p->prof_events[i].data();
    BG_CUDA(cudaEventSynchronize(ev[3]), "profiling event sync");
    float a = 0, b = 0, c = 0;
    BG_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]), "profiling elapsed");
    BG_CUDA(cudaEventElapsedTime(&c, ev[1], ev[2]), "profiling elapsed");
    BG_CUDA(cudaEventElapsedTime(&b, ev[2], ev[3]), "profiling elapsed");
    p->prof_ms[0] += a;
    p->prof_ms[1] += b;
    p->prof_ms[2] += c;
    p->prof_calls++;
  }
  p->prof_used = 0;
  for (int i = 0; i < 3; ++i) total_ms[i] = p->prof_ms[i];
  *calls = p->prof_calls;
  if (reset) {
    p->prof_ms[0] = p->prof_ms[1] = p->prof_ms[2] = 0.0;
    p->prof_calls = 0;
  }
  return BG_OK;
}

bg_status bg_plan_get_info(const bg_plan* p, bg_plan_info* out) {
  if (!p || !out) return fail(BG_ERR_INVALID_ARG, "null pointer");
  out->count = p->count;
  out->work_items = (p->split ? split_plan_items(p->split) : 0) + p->n_items;
  out->launches_per_call = p->launches_per_call;
  out->classes = (int32_t)p->classes.size();
  out->workspace_bytes = p->workspace_bytes;
  out->slices = p->prec.mode == BG_MODE_SPLIT_BF16 ? p->prec.slices : 0;
  out->beta_bits = p->split ? split_plan_beta_bits(p->split) : 0;
  return BG_OK;
}

bg_status bg_plan_describe(const bg_plan* p, char* buf, size_t len, size_t* needed) {
  if (!p) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
  static const char* names[] = {"r64_small_warp", "r64_tile64_dfma", "r64_tile64_dmma",
                                "c128_small_warp", "c128_tile32_dfma"};
  std::string s = "{\"dtype\": \"";
  s += p->dtype == BG_C128 ? "c128" : "r64";
  s += "\", \"mode\": \"";
  s += p->prec.mode == BG_MODE_FP64 ? "fp64" : "split_bf16";
  s += "\", \"classes\": [";
  for (size_t c = 0; c < p->classes.size(); ++c) {
    const ClassInfo& ci = p->classes[c];
    char tmp[512];
    snprintf(tmp, sizeof tmp,
             "%s{\"bucket\": [%lld, %lld, %lld], \"members\": %lld, \"gflop\": %.6f, "
             "\"program\": \"%s\", \"timed_ms\": %.6f, \"tried\": [",
             c ? ", " : "", (long long)ci.key_m, (long long)ci.key_n, (long long)ci.key_k,
             (long long)ci.members, ci.flops * 1e-9,
             (ci.prog >= 0 && ci.prog < PROG_COUNT) ? names[ci.prog] : split_route_name(ci.prog),
             ci.ms);
    s += tmp;
    for (size_t t = 0; t < ci.tried.size(); ++t) {
      const int q = ci.tried[t].first;
      snprintf(tmp, sizeof tmp, "%s{\"program\": \"%s\", \"ms\": %.6f}", t ? ", " : "",
               (q >= 0 && q < PROG_COUNT) ? names[q] : split_route_name(q), ci.tried[t].second);
      s += tmp;
    }
    s += "]}";
  }
  s += "]";
  if (p->split) s += ", \"split\": " + split_plan_describe(p->split);
  s += "}";
  if (needed) *needed = s.size() + 1;
  if (!buf || len < s.size() + 1) return fail(BG_ERR_INVALID_ARG, "buffer too small");
  memcpy(buf, s.c_str(), s.size() + 1);
  return BG_OK;
}

bg_status bg_rel_err(bg_dtype dtype, int64_t count, const int64_t* d_table, const void* A,
                     const void* B, const void* C_test, const void* C_ref, double* d_out,
                     bg_stream_t stream) {
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  if (count < 0) return fail(BG_ERR_INVALID_ARG, "negative count");
  if (count == 0) return BG_OK;
  if (!d_table || !A || !B || !C_test || !C_ref || !d_out)
    return fail(BG_ERR_INVALID_ARG, "null pointer");
  cudaError_t e = launch_rel_err(dtype, count, d_table, A, B, C_test, C_ref, d_out,
                                 reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rel_err launch");
  return BG_OK;
}

bg_status bg_unitarity_drift(bg_dtype dtype, int64_t count, const int64_t* d_n,
                             const int64_t* d_off, const void* C, double* d_out,
                             bg_stream_t stream) {
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  if (count < 0) return fail(BG_ERR_INVALID_ARG, "negative count");
  if (count == 0) return BG_OK;
  if (!d_n || !d_off || !C || !d_out) return fail(BG_ERR_INVALID_ARG, "null pointer");
  cudaError_t e = launch_drift(dtype, count, d_n, d_off, C, d_out,
                               reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "drift launch");
  return BG_OK;
}

bg_status apply_local_gate(bg_dtype dtype, int64_t walkers, int32_t spins, const int32_t* sites,
                           const void* gates, void* states, int64_t stride, bg_stream_t stream) {
  bg_status s = check_dtype(dtype);
  if (s != BG_OK) return s;
  if (dtype != BG_C128) return fail(BG_ERR_UNSUPPORTED, "the local gate acts on complex128 states");
  if (walkers < 0) return fail(BG_ERR_INVALID_ARG, "negative walker count");
  if (spins < 2 || spins > 40) return fail(BG_ERR_INVALID_ARG, "spins must be 2..40");
  if (stride < ((int64_t)1 << spins))
    return fail(BG_ERR_INVALID_ARG, "stride below 2^spins amplitudes");
  if (walkers == 0) return BG_OK;
  if (!sites || !gates || !states) return fail(BG_ERR_INVALID_ARG, "null pointer");
  if (!aligned(gates, BG_C128) || !aligned(states, BG_C128))
    return fail(BG_ERR_INVALID_ARG, "gates or states not 16-byte aligned");
  DeviceCtx* ctx;
  s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  cudaError_t e = launch_local_gate(walkers, spins, sites, gates, states, stride, ctx->d_err,
                                    ctx->sms, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "local gate launch");
  return BG_OK;
}

bg_status bg_split_planes(int64_t m, int64_t k, const double* X, int64_t ldx, int32_t axis,
                          int32_t slices, int32_t beta_bits, int32_t* exps, uint16_t* digits,
                          bg_stream_t stream) {
  if (m < 0 || k < 0) return fail(BG_ERR_INVALID_ARG, "negative size");
  if (ldx < std::max<int64_t>(1, m)) return fail(BG_ERR_INVALID_ARG, "ldx below the row count");
  if (axis != 0 && axis != 1) return fail(BG_ERR_INVALID_ARG, "axis must be 0 or 1");
  if (slices < 1 || slices > kMaxSlices)
    return fail(BG_ERR_INVALID_ARG, "slices must be 1..%d", kMaxSlices);
  if (beta_bits < 2 || beta_bits > 8) return fail(BG_ERR_INVALID_ARG, "beta_bits must be 2..8");
  if (m == 0 || k == 0) return BG_OK;
  if (!X || !exps || !digits) return fail(BG_ERR_INVALID_ARG, "null pointer");
  if (!aligned(X, BG_R64)) return fail(BG_ERR_INVALID_ARG, "X misaligned");
  cudaError_t e = launch_split_planes(m, k, X, ldx, axis, slices, beta_bits, exps, digits,
                                      reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "split planes launch");
  return BG_OK;
}

bg_status bg_check_device_errors(bg_stream_t stream) {
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BG_CUDA(cudaStreamSynchronize(st), "stream synchronize");
  int h[4] = {0, 0, 0, 0};
  BG_CUDA(cudaMemcpy(h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost), "read error word");
  BG_CUDA(cudaMemset(ctx->d_err, 0, sizeof h), "clear error word");
  if (h[0] != 0)
    return fail((bg_status)h[0], "device error %d at location %d (detail %d, %d event(s))", h[0],
                h[1], h[2], h[3]);
  return BG_OK;
}

bg_status bg_test_bounded_wait(int64_t spin_limit, bg_stream_t stream) {
  if (spin_limit < 1 || spin_limit > (int64_t)1 << 40)
    return fail(BG_ERR_INVALID_ARG, "spin_limit out of range");
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  cudaError_t e = launch_bounded_wait(spin_limit, ctx->d_err, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bounded wait launch");
  return BG_OK;
}

bg_status bg_probe_fp64_peak(int32_t mma_kind, double* tflops, bg_stream_t stream) {
  if (!tflops) return fail(BG_ERR_INVALID_ARG, "tflops is NULL");
  if (mma_kind != 0 && mma_kind != 1) return fail(BG_ERR_INVALID_ARG, "mma_kind must be 0 or 1");
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  cudaError_t e = run_fp64_peak_probe(mma_kind, ctx->sms, tflops,
                                      reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "FP64 peak probe");
  return BG_OK;
}

bg_status entropy_plan(bg_plan** out, int64_t walkers, int32_t spins, int32_t split,
                       int64_t stride, const bg_precision* precision, uint32_t flags,
                       bg_stream_t stream) {
  if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  bg_precision pr;
  bg_status s = check_precision(precision, &pr);
  if (s != BG_OK) return s;
  if (walkers < 0 || walkers > 65535)
    return fail(BG_ERR_INVALID_ARG, "walkers = %lld outside 0..65535", (long long)walkers);
  if (spins < 2 || spins > 30) return fail(BG_ERR_INVALID_ARG, "spins = %d outside 2..30", spins);
  if (split < 1 || split > spins - 1 || split > 10)
    return fail(BG_ERR_INVALID_ARG, "split = %d outside 1..min(spins - 1, 10)", split);
  if (stride < ((int64_t)1 << spins))
    return fail(BG_ERR_INVALID_ARG, "stride %lld below 2^spins", (long long)stride);
  if (flags & ~(uint32_t)BG_PLAN_PROFILE)
    return fail(BG_ERR_INVALID_ARG, "entropy plans take BG_PLAN_PROFILE only");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (stream_capturing(st))
    return fail(BG_ERR_CAPTURE, "entropy_plan allocates; the stream is being captured");
  DeviceCtx* ctx;
  if ((s = get_ctx(&ctx)) != BG_OK) return s;
  const int64_t K = (int64_t)1 << split, M = (int64_t)1 << (spins - split);
  // walker w: X = its state as a column-major K x M matrix; G = X X^H (K x K)
  std::vector<bg_instance> table((size_t)walkers);
  for (int64_t w = 0; w < walkers; ++w)
    table[(size_t)w] = bg_instance{K, K, M, K, M, K, w * stride, 0, w * K * K};
  bg_plan* p = new bg_plan();
  p->device = ctx->device;
  p->dtype = BG_C128;
  p->prec = pr;
  p->flags = flags;
  p->count = walkers;
  p->is_entropy = true;
  p->ent_n = (int)K;
  if (walkers > 0) {
    s = batched_gemm_plan(&p->gram, BG_C128, walkers, table.data(), &pr, BG_PLAN_HERK, nullptr,
                          stream);
    if (s != BG_OK) {
      destroy_plan(p);
      return s;
    }
    const size_t gb = (size_t)walkers * K * K * sizeof(double2);
    const size_t tb = (size_t)walkers * K * sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_gram, gb)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_tri_d, tb)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_tri_e, tb)) != cudaSuccess) {
      destroy_plan(p);
      return cuda_fail(e, "entropy plan workspace");
    }
    p->workspace_bytes = p->gram->workspace_bytes + (int64_t)(gb + 2 * tb);
    p->launches_per_call = p->gram->launches_per_call + 2;
    if (pr.mode != BG_MODE_FP64 && K > kTriTail) {
      // blocked reduction: panels of nb columns while more than kTriTail
      // columns remain, each followed by its trailing update in the plan's
      // precision; the last kTriTail columns are reduced unblocked
      const int nb = kTriPanelWidth;
      const int64_t pstride = 2 * (int64_t)nb * K;
      const size_t pb = (size_t)walkers * pstride * sizeof(double2);
      const size_t wb = (size_t)walkers * (K - nb) * 2 * nb * sizeof(double2);
      const size_t sb = (size_t)walkers * K * K * sizeof(double);
      if ((e = cudaMalloc(&p->d_tri_p, pb)) != cudaSuccess ||
          (e = cudaMalloc(&p->d_tri_wvh, wb)) != cudaSuccess ||
          (e = cudaMalloc(&p->d_tri_s, sb)) != cudaSuccess) {
        destroy_plan(p);
        return cuda_fail(e, "entropy plan workspace");
      }
      p->tri_nb = nb;
      p->tri_pstride = pstride;
      p->workspace_bytes += (int64_t)(pb + wb + sb);
      p->launches_per_call = p->gram->launches_per_call + 3;  // mirror, tail, bisection
      for (int64_t p0 = 0; K - p0 > kTriTail; p0 += nb) {
        const int64_t q = p0 + nb, mt = K - q;
        for (int64_t w = 0; w < walkers; ++w)
          table[(size_t)w] = bg_instance{mt, mt, 2 * nb, K, 2 * nb, K, w * pstride + q,
                                         w * mt * 2 * nb, w * K * K + q + q * K};
        bg_plan* g = nullptr;
        s = batched_gemm_plan(&g, BG_C128, walkers, table.data(), &pr, 0, nullptr, stream);
        if (s != BG_OK) {
          destroy_plan(p);
          return s;
        }
        p->tri_gemm.push_back(g);
        p->workspace_bytes += g->workspace_bytes;
        p->launches_per_call += 3 + g->launches_per_call;  // panel, pack, GEMM, sum
      }
    }
  }
  *out = p;
  return BG_OK;
}

bg_status batched_entropy(const bg_plan* plan, const void* states, double* entropy,
                          double* eigenvalues, bg_stream_t stream) {
  if (!plan) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->is_entropy) return fail(BG_ERR_INVALID_ARG, "not an entropy plan");
  if (plan->count == 0) return BG_OK;
  if (!states || !entropy) return fail(BG_ERR_INVALID_ARG, "null device pointer");
  if (reinterpret_cast<uintptr_t>(states) % 16 != 0)
    return fail(BG_ERR_INVALID_ARG, "states must be 16-byte aligned");
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch failure (BGEMM_FAULT)");
  bg_plan* p = const_cast<bg_plan*>(plan);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t* ev = nullptr;
  if (p->flags & BG_PLAN_PROFILE) {
    if (p->prof_used == p->prof_events.size()) {
      std::array<cudaEvent_t, 4> tev{};
      for (auto& e : tev) BG_CUDA(cudaEventCreate(&e), "profiling event");
      p->prof_events.push_back(tev);
    }
    ev = p->prof_events[p->prof_used++].data();
    BG_CUDA(cudaEventRecord(ev[0], st), "profiling event record");
  }
  const double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0};
  bg_status s = batched_gemm_grouped(p->gram, states, nullptr, p->d_gram, one, zero, stream);
  if (s != BG_OK) return s;
  if (ev) {
    BG_CUDA(cudaEventRecord(ev[1], st), "profiling event record");
    BG_CUDA(cudaEventRecord(ev[2], st), "profiling event record");
  }
  if (p->tri_gemm.empty()) {
    cudaError_t e = launch_entropy_eig(p->d_gram, p->count, p->ent_n, p->d_tri_d, p->d_tri_e,
                                       entropy, eigenvalues, st);
    if (e != cudaSuccess) return cuda_fail(e, "entropy eigenvalue launch");
  } else {
    const int n = p->ent_n, nb = p->tri_nb;
    const double minus_one[2] = {-1.0, 0.0};
    cudaError_t e0 = launch_tri_mirror(p->d_gram, p->d_tri_s, p->count, n, st);
    if (e0 != cudaSuccess) return cuda_fail(e0, "entropy mirror launch");
    int p0 = 0;
    for (bg_plan* g : p->tri_gemm) {
      cudaError_t e = launch_tri_panel(p->d_gram, p->d_tri_s, p->count, n, p0, nb, p->d_tri_p,
                                       p->tri_pstride, p->d_tri_d, p->d_tri_e, st);
      if (e == cudaSuccess)
        e = launch_tri_pack(p->d_tri_p, p->tri_pstride, p->count, n, p0 + nb, nb, p->d_tri_wvh,
                            st);
      if (e != cudaSuccess) return cuda_fail(e, "entropy panel launch");
      s = batched_gemm_grouped(g, p->d_tri_p, p->d_tri_wvh, p->d_gram, minus_one, one, stream);
      if (s != BG_OK) return s;
      e = launch_tri_sum(p->d_gram, p->d_tri_s, p->count, n, p0 + nb, st);
      if (e != cudaSuccess) return cuda_fail(e, "entropy panel launch");
      p0 += nb;
    }
    cudaError_t e = launch_tri_tail(p->d_gram, p->count, n, p0, p->d_tri_d, p->d_tri_e, st);
    if (e == cudaSuccess)
      e = launch_entropy_bisect(p->d_tri_d, p->d_tri_e, p->count, n, entropy, eigenvalues, st);
    if (e != cudaSuccess) return cuda_fail(e, "entropy eigenvalue launch");
  }
  if (ev) BG_CUDA(cudaEventRecord(ev[3], st), "profiling event record");
  return BG_OK;
}

bg_status metropolis_select(int64_t walkers, double temperature, int32_t direction,
                            const double* uniforms, const double* e_new, double* e_cur,
                            int32_t* accepted, const void* proposals, int64_t proposal_stride,
                            void* states, int64_t state_stride, int64_t amplitudes,
                            bg_stream_t stream) {
  if (walkers < 0) return fail(BG_ERR_INVALID_ARG, "negative walker count");
  if (!(temperature >= 0.0)) return fail(BG_ERR_INVALID_ARG, "temperature must be >= 0");
  if (direction != 1 && direction != -1) return fail(BG_ERR_INVALID_ARG, "direction must be +1 or -1");
  if (amplitudes < 0) return fail(BG_ERR_INVALID_ARG, "negative amplitude count");
  if (walkers == 0) return BG_OK;
  if (!uniforms || !e_new || !e_cur || !accepted)
    return fail(BG_ERR_INVALID_ARG, "null device pointer");
  if (amplitudes > 0) {
    if (!proposals || !states) return fail(BG_ERR_INVALID_ARG, "null state pointer");
    if (proposal_stride < amplitudes || state_stride < amplitudes)
      return fail(BG_ERR_INVALID_ARG, "strides below the amplitude count");
    if (!aligned(proposals, BG_C128) || !aligned(states, BG_C128))
      return fail(BG_ERR_INVALID_ARG, "states not 16-byte aligned");
  }
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch failure (BGEMM_FAULT)");
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  cudaError_t e = launch_metropolis(walkers, temperature, direction, uniforms, e_new, e_cur,
                                    accepted, proposals, proposal_stride, states, state_stride,
                                    amplitudes, ctx->sms, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "Metropolis launch");
  return BG_OK;
}

bg_status anneal_plan(bg_plan** out, int64_t walkers, int32_t spins, int32_t split,
                      int64_t stride, const bg_precision* precision, uint32_t flags,
                      bg_stream_t stream) {
  if (!out) return fail(BG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (flags & ~(uint32_t)BG_PLAN_PROFILE)
    return fail(BG_ERR_INVALID_ARG, "annealing plans take BG_PLAN_PROFILE only");
  bg_plan* ent = nullptr;
  const int64_t amps = spins >= 2 && spins <= 30 ? (int64_t)1 << spins : 0;
  // the entropy plan checks walkers, spins, split and the precision
  bg_status s = entropy_plan(&ent, walkers, spins, split, amps, precision, flags, stream);
  if (s != BG_OK) return s;
  if (stride < amps) {
    destroy_plan(ent);
    return fail(BG_ERR_INVALID_ARG, "stride %lld below 2^spins", (long long)stride);
  }
  bg_plan* p = new bg_plan();
  p->device = ent->device;
  p->dtype = BG_C128;
  p->prec = ent->prec;
  p->flags = flags;
  p->count = walkers;
  p->is_anneal = true;
  p->ent = ent;
  p->spins = spins;
  p->state_stride = stride;
  if (walkers > 0) {
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_prop, (size_t)walkers * amps * sizeof(double2))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_enew, (size_t)walkers * sizeof(double))) != cudaSuccess) {
      destroy_plan(p);
      return cuda_fail(e, "annealing plan workspace");
    }
  }
  p->workspace_bytes = ent->workspace_bytes + walkers * (amps * (int64_t)sizeof(double2) + 8);
  p->launches_per_call = 1 + ent->launches_per_call + 2;
  *out = p;
  return BG_OK;
}

bg_status anneal_step(const bg_plan* plan, void* states, double* energy, const int32_t* sites,
                      const void* gates, const double* uniforms, double temperature,
                      int32_t direction, int32_t* accepted, bg_stream_t stream) {
  if (!plan) return fail(BG_ERR_INVALID_ARG, "plan is NULL");
  if (!plan->is_anneal) return fail(BG_ERR_INVALID_ARG, "not an annealing plan");
  if (plan->count == 0) return BG_OK;
  if (!states || !energy || !sites || !gates || !uniforms || !accepted)
    return fail(BG_ERR_INVALID_ARG, "null device pointer");
  if (!aligned(states, BG_C128) || !aligned(gates, BG_C128))
    return fail(BG_ERR_INVALID_ARG, "states or gates not 16-byte aligned");
  if (!(temperature >= 0.0)) return fail(BG_ERR_INVALID_ARG, "temperature must be >= 0");
  if (direction != 1 && direction != -1) return fail(BG_ERR_INVALID_ARG, "direction must be +1 or -1");
  if (fault_injected()) return fail(BG_ERR_CUDA, "injected launch failure (BGEMM_FAULT)");
  bg_plan* p = const_cast<bg_plan*>(plan);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t amps = (int64_t)1 << p->spins;
  DeviceCtx* ctx;
  bg_status s = get_ctx(&ctx);
  if (s != BG_OK) return s;
  // 1. the proposal: a copy of every current state ...
  BG_CUDA(cudaMemcpy2DAsync(p->d_prop, amps * sizeof(double2), states,
                            p->state_stride * sizeof(double2), amps * sizeof(double2), p->count,
                            cudaMemcpyDeviceToDevice, st),
          "proposal copy");
  // 2. ... with the walker's local gate applied ("Apply Local Gate")
  cudaError_t e = launch_local_gate(p->count, p->spins, sites, gates, p->d_prop, amps, ctx->d_err,
                                    ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "local gate launch");
  // 3. its entanglement entropy ("Calculate Entropy")
  if ((s = batched_entropy(p->ent, p->d_prop, p->d_enew, nullptr, stream)) != BG_OK) return s;
  // 4. the Metropolis decision ("M.A"): accepted proposals replace the states
  e = launch_metropolis(p->count, temperature, direction, uniforms, p->d_enew, energy, accepted,
                        p->d_prop, amps, states, p->state_stride, amps, ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "Metropolis launch");
  return BG_OK;
}

bg_status bg_partition_lpt(int64_t count, const double* host_cost, int32_t parts,
                           int32_t* out_part, double* out_load) {
  if (count < 0) return fail(BG_ERR_INVALID_ARG, "negative count");
  if (parts < 1) return fail(BG_ERR_INVALID_ARG, "parts must be >= 1");
  if (count > 0 && (!host_cost || !out_part))
    return fail(BG_ERR_INVALID_ARG, "host_cost and out_part must not be NULL");
  for (int64_t i = 0; i < count; ++i)
    if (!(host_cost[i] >= 0.0) || std::isinf(host_cost[i]))
      return fail(BG_ERR_INVALID_ARG, "cost %lld is negative or not finite", (long long)i);
  // longest first; equal costs keep the lower index first
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return host_cost[a] > host_cost[b]; });
  // min-heap of (load, part): the least loaded part, the lower index on ties
  using Slot = std::pair<double, int32_t>;
  std::vector<Slot> heap;
  heap.reserve((size_t)parts);
  for (int32_t r = 0; r < parts; ++r) heap.push_back({0.0, r});
  auto later = [](const Slot& a, const Slot& b) {
    return a.first > b.first || (a.first == b.first && a.second > b.second);
  };
  std::make_heap(heap.begin(), heap.end(), later);
  std::vector<double> load((size_t)parts, 0.0);
  for (int64_t i : order) {
    std::pop_heap(heap.begin(), heap.end(), later);
    Slot s = heap.back();
    out_part[i] = s.second;
    s.first += host_cost[i];
    load[(size_t)s.second] = s.first;
    heap.back() = s;
    std::push_heap(heap.begin(), heap.end(), later);
  }
  if (out_load)
    for (int32_t r = 0; r < parts; ++r) out_load[r] = load[(size_t)r];
  return BG_OK;
}

int64_t bg_launch_count(int32_t reset) {
  const int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

const char* bg_status_string(bg_status s) {
  switch (s) {
    case BG_OK: return "BG_OK";
    case BG_ERR_INVALID_ARG: return "BG_ERR_INVALID_ARG";
    case BG_ERR_UNSUPPORTED: return "BG_ERR_UNSUPPORTED";
    case BG_ERR_CUDA: return "BG_ERR_CUDA";
    case BG_ERR_NOMEM: return "BG_ERR_NOMEM";
    case BG_ERR_CAPTURE: return "BG_ERR_CAPTURE";
    case BG_ERR_TIMEOUT: return "BG_ERR_TIMEOUT";
    default: return "BG_ERR_UNKNOWN";
  }
}

const char* bg_last_error(void) { return g_last_error.c_str(); }

const char* bg_version(void) { return "bgemm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
