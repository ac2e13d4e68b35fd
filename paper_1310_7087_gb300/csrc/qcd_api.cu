// qcd_api.cu -- host side of libqcdgb300: the C ABI declared in include/qcd.h.
// Lattice objects, argument checks, the sweep schedule (captured once per
// (seed, n_or, nhit, block) into a CUDA graph), the launch-shape autotuner and
// host <-> device copies.  Every step of the sweep and of the measurements runs
// in the kernels of su{2,3}_f{32,64}.cu.
#include "qcd.h"
#include "qcd_internal.h"
#include "qcd_split.h"

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace {

thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define QCD_CUDA(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return set_error(QCD_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                       __LINE__);                                                                        \
  } while (0)

struct GraphKey {
  uint64_t seed;
  int n_or, nhit, block, profiled, measured, instance;
  bool operator==(const GraphKey& o) const {
    return seed == o.seed && n_or == o.n_or && nhit == o.nhit && block == o.block && profiled == o.profiled &&
           measured == o.measured && instance == o.instance;
  }
};

// A captured sweep.  When profiled, events[k], events[k + 1] bracket group k
// of counts[k] kernels of category kinds[k]; `pending` marks a launch whose
// events have not been read yet.  Two instances of a profiled graph alternate,
// so reading one launch's events waits for the launch before the previous one
// (normally long finished) and the sweeps stay queued back to back.
struct SweepGraph {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;
  std::vector<int> kinds;
  std::vector<int> counts;
  bool pending = false;
};

// Process-wide autotune cache: (group, precision, Ns, Nt, field, device) ->
// threads per block of the phase kernels.  Persisted to the file named by
// QCD_AUTOTUNE_CACHE when that variable is set.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
  const char* p = getenv("QCD_AUTOTUNE_CACHE");
  return p ? std::string(p) : std::string();
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const std::string path = tune_path();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  char key[256];
  int block;
  while (fscanf(f, "%255s %d", key, &block) == 2) g_tune[key] = block;
  fclose(f);
}

void tune_store_locked() {
  const std::string path = tune_path();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "w");
  if (!f) return;
  for (const auto& kv : g_tune) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
  fclose(f);
}

}  // namespace

struct qcd_lattice {
  const qcd::PolicyOps* ops = nullptr;
  int group = 0, precision = 0, Ns = 0, Nt = 0, flux = 0, flux8 = 0, nhit = 10;
  int field_mode = QCD_FIELD_LINKS;
  double beta = 0.0;
  uint64_t seed = 0;
  uint32_t lattice_id = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int block = 0;  // threads per block of the phase kernels; 0 = autotune
  qcd::GeomH g{};
  void* links = nullptr;
  size_t link_bytes = 0;
  qcd::SplitLinks* split = nullptr;  // non-null: links divided between device and host memory
  size_t split_device_bytes = 0;     // device-resident bytes of each link array
  unsigned char* d_small = nullptr;  // sweep counter, exhaustion counter, results
  uint32_t* d_sweep = nullptr;
  unsigned long long* d_exhausted = nullptr;
  double* d_meas = nullptr;
  double* d_partials = nullptr;
  double2* d_phase64 = nullptr;  // 4 Ns entries: lambda3 phase, then the SU(3) diagonal
  float2* d_phase32 = nullptr;
  std::vector<SweepGraph> graphs;
  int profiling = 0;
  int prof_flip = 0;  // alternates the two instances of a profiled graph
  double prof_ms[QCD_PROF_N] = {0, 0, 0, 0};
  unsigned long long prof_launches[QCD_PROF_N] = {0, 0, 0, 0};
  cudaEvent_t meas_ev[2] = {nullptr, nullptr};
};

namespace {

__global__ void phase_table_kernel(double2* p64, float2* p32, int Ns, int flux, int flux8) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Ns) return;
  // phi = 2 pi n x / Ns^2, as sincospi of 2 n x / Ns^2 (exact argument reduction)
  const double unit = 2.0 * double(x) / (double(Ns) * double(Ns));
  double s, c;
  sincospi(double(flux) * unit, &s, &c);
  p64[x] = make_double2(c, s);
  p32[x] = make_float2(float(c), float(s));
  // SU(3) diagonal: theta = 2 pi x / Ns^2 (n + n8, -n + n8, -2 n8)
  const int h[3] = {flux + flux8, -flux + flux8, -2 * flux8};
  for (int k = 0; k < 3; ++k) {
    sincospi(double(h[k]) * unit, &s, &c);
    p64[Ns + 3 * x + k] = make_double2(c, s);
    p32[Ns + 3 * x + k] = make_float2(float(c), float(s));
  }
}

const qcd::PolicyOps* pick_ops(int group, int precision) {
  if (group == 2) return precision == QCD_FP64_PLAIN ? &qcd::kOpsSU2F64 : &qcd::kOpsSU2F32;
  return precision == QCD_FP64_PLAIN ? &qcd::kOpsSU3F64 : &qcd::kOpsSU3F32;
}

qcd::Ctx make_ctx(const qcd_lattice* L, uint64_t seed) {
  qcd::Ctx a{};
  a.links = L->links;
  a.g = L->g;
  a.beta = L->beta;
  a.k0 = uint32_t(seed) ^ (L->lattice_id * 0x9E3779B9u);
  a.k1 = uint32_t(seed >> 32);
  a.sweep = L->d_sweep;
  a.sweep_rw = L->d_sweep;
  a.nhit = L->nhit;
  a.flux = L->flux;
  a.field_mode = L->field_mode;
  a.phase64 = L->d_phase64;
  a.phase32 = L->d_phase32;
  a.flux8 = L->flux8;
  a.exhausted = L->d_exhausted;
  a.partials = L->d_partials;
  a.meas_out = L->d_meas;
  return a;
}

int check(const qcd_lattice* L) {
  if (!L) return set_error(QCD_ERR_INVALID_ARG, "null lattice handle");
  return QCD_OK;
}

int use_device(const qcd_lattice* L) {
  int cur = -1;
  QCD_CUDA(cudaGetDevice(&cur));
  if (cur != L->device) QCD_CUDA(cudaSetDevice(L->device));
  return QCD_OK;
}

void drop_graph(SweepGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (cudaEvent_t e : g.events) cudaEventDestroy(e);
  g.exec = nullptr;
  g.events.clear();
}

void drop_graphs(qcd_lattice* L) {
  for (auto& g : L->graphs) drop_graph(g);
  L->graphs.clear();
}

__global__ void sweep_advance_kernel(uint32_t* sweep) { *sweep += 1u; }

// One sweep: heat-bath pass, n_or overrelaxation passes, reunitarization, and
// the advance of the sweep counter.  The reunitarization rides on the last
// overrelaxation pass (each link is updated once in a pass; that pass's
// kernels reunitarize it before the store), so no separate pass over the
// links is needed; with n_or = 0 the reunitarization kernel runs.  With
// events, event k is recorded before kernel k and the last one after the
// final kernel.
int enqueue_sweep(const qcd_lattice* L, const qcd::Ctx& a, int n_or, int block, bool measured, cudaStream_t st,
                  const std::vector<cudaEvent_t>* events) {
  size_t k = 0;
  // External event-record nodes: the events stay usable (synchronize, elapsed
  // time) after every launch of the captured graph.
  auto mark = [&]() -> cudaError_t {
    return events ? cudaEventRecordWithFlags((*events)[k++], st, cudaEventRecordExternal) : cudaSuccess;
  };
  // event groups: heat-bath pass | overrelaxation passes but the last | last
  // pass and the counter advance (or the reunitarization kernel) | measurement tail
  QCD_CUDA(mark());
  for (int p = 0; p < 2; ++p)
    for (int mu = 0; mu < 4; ++mu) QCD_CUDA(L->ops->phase(a, qcd::KIND_HB, p, mu, block, st));
  for (int o = 0; o < n_or; ++o) {
    if (o == 0 && n_or > 1) QCD_CUDA(mark());
    if (o == n_or - 1) QCD_CUDA(mark());
    for (int p = 0; p < 2; ++p)
      for (int mu = 0; mu < 4; ++mu) {
        const int kind = o < n_or - 1 ? qcd::KIND_OR
                         : (measured && p == 1 && mu >= 1) ? qcd::KIND_OR_MEAS : qcd::KIND_OR_REUNIT;
        QCD_CUDA(L->ops->phase(a, kind, p, mu, block, st));
      }
  }
  if (n_or == 0) QCD_CUDA(mark());
  if (n_or > 0) {
    sweep_advance_kernel<<<1, 1, 0, st>>>(a.sweep_rw);
    QCD_CUDA(cudaGetLastError());
  } else {
    QCD_CUDA(L->ops->reunit(a, 1, st));  // no overrelaxation pass to carry it
  }
  QCD_CUDA(mark());
  if (measured) {  // Polyakov loop and the final sums of the fused measurement
    QCD_CUDA(L->ops->measure_fused_tail(a, block, st));
    QCD_CUDA(mark());
  }
  return QCD_OK;
}

int fold_all(qcd_lattice* L);

int get_graph(qcd_lattice* L, uint64_t seed, int n_or, bool measured, SweepGraph** out) {
  const int instance = L->profiling ? (L->prof_flip ^= 1) : 0;
  const GraphKey key{seed, n_or, L->nhit, L->block, L->profiling, measured ? 1 : 0, instance};
  for (auto& g : L->graphs)
    if (g.key == key) {
      *out = &g;
      return QCD_OK;
    }
  if (L->graphs.size() >= 8) {
    if (int rc = fold_all(L)) return rc;  // keep the profile of launches in flight
    drop_graphs(L);
  }
  SweepGraph sg;
  sg.key = key;
  if (L->profiling) {
    // buckets: heat-bath pass; overrelaxation passes but the last; the last
    // pass (it carries the reunitarization) and the counter advance
    sg.kinds.push_back(QCD_PROF_HEATBATH);
    sg.counts.push_back(8);
    if (n_or > 1) {
      sg.kinds.push_back(QCD_PROF_OVERRELAX);
      sg.counts.push_back(8 * (n_or - 1));
    }
    sg.kinds.push_back(QCD_PROF_REUNIT);
    sg.counts.push_back(n_or > 0 ? 9 : 1);
    if (measured) {
      sg.kinds.push_back(QCD_PROF_MEASURE);
      sg.counts.push_back(2);
    }
    sg.events.resize(sg.kinds.size() + 1, nullptr);
    for (auto& e : sg.events)
      if (cudaEventCreate(&e) != cudaSuccess) {
        drop_graph(sg);
        return set_error(QCD_ERR_CUDA, "cudaEventCreate failed");
      }
  }
  cudaStream_t cap;
  QCD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const qcd::Ctx a = make_ctx(L, seed);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = QCD_OK;
  if (e == cudaSuccess) {
    rc = enqueue_sweep(L, a, n_or, L->block, measured, cap, L->profiling ? &sg.events : nullptr);
    e = cudaStreamEndCapture(cap, &graph);
  }
  cudaStreamDestroy(cap);
  if (rc != QCD_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    drop_graph(sg);
    return rc != QCD_OK ? rc : set_error(QCD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&sg.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    drop_graph(sg);
    return set_error(QCD_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  L->graphs.push_back(sg);
  *out = &L->graphs.back();
  return QCD_OK;
}

// Add the durations bracketed by a completed profiled graph's events.
int fold_profile(qcd_lattice* L, SweepGraph& g) {
  if (!g.pending) return QCD_OK;
  g.pending = false;
  QCD_CUDA(cudaEventSynchronize(g.events.back()));
  for (size_t k = 0; k + 1 < g.events.size(); ++k) {
    float ms = 0.f;
    QCD_CUDA(cudaEventElapsedTime(&ms, g.events[k], g.events[k + 1]));
    L->prof_ms[g.kinds[k]] += ms;
    L->prof_launches[g.kinds[k]] += g.counts[k];
  }
  return QCD_OK;
}

int fold_all(qcd_lattice* L) {
  for (auto& g : L->graphs)
    if (int rc = fold_profile(L, g)) return rc;
  return QCD_OK;
}

// Launch a captured sweep; a profiled one first reads the events of this
// instance's previous launch.
int launch_graph(qcd_lattice* L, SweepGraph& g) {
  if (int rc = fold_profile(L, g)) return rc;
  QCD_CUDA(cudaGraphLaunch(g.exec, L->stream));
  g.pending = L->profiling != 0;
  return QCD_OK;
}

std::string tune_key(const qcd_lattice* L) {
  cudaDeviceProp prop;
  std::string dev = "gpu";
  if (cudaGetDeviceProperties(&prop, L->device) == cudaSuccess) {
    dev = prop.name;
    for (auto& ch : dev)
      if (ch == ' ') ch = '_';
  }
  char buf[256];
  snprintf(buf, sizeof buf, "su%d_p%d_%dx%d_f%d_%s", L->group, L->precision, L->Ns, L->Nt,
           L->field_mode != QCD_FIELD_LINKS ? 0 : L->flux8 != 0 ? 2 : L->flux != 0 ? 1 : 0,
           dev.c_str());
  return buf;
}

// Time one heat-bath and one overrelaxation phase for each candidate block
// size on a scratch copy of the links, keep the fastest.  The lattice state and
// counters are not touched.
int autotune(qcd_lattice* L) {
  const std::string key = tune_key(L);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      L->block = it->second;
      return QCD_OK;
    }
  }
  const char* env = getenv("QCD_AUTOTUNE");
  if ((env && env[0] == '0') || L->split) {  // a split lattice may not fit a device scratch copy
    L->block = 128;
    return QCD_OK;
  }
  void* scratch = nullptr;
  unsigned long long* dummy = nullptr;
  QCD_CUDA(cudaMallocAsync(&scratch, L->link_bytes, L->stream));
  QCD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dummy), sizeof(unsigned long long), L->stream));
  QCD_CUDA(cudaMemcpyAsync(scratch, L->links, L->link_bytes, cudaMemcpyDeviceToDevice, L->stream));
  qcd::Ctx a = make_ctx(L, L->seed);
  a.links = scratch;
  a.exhausted = dummy;
  cudaEvent_t e0, e1;
  QCD_CUDA(cudaEventCreate(&e0));
  QCD_CUDA(cudaEventCreate(&e1));
  const int cand[] = {64, 128, 256, 512};
  const int limit = L->ops->max_phase_block();
  int best = 0;
  float best_ms = 1e30f;
  for (int c = 0; c < 4; ++c) {
    const int b = cand[c];
    if (b > limit) continue;  // more registers than the SM gives one block
    // one warm-up round, then two timed rounds
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      if (rep == 1) cudaEventRecord(e0, L->stream);
      ok = L->ops->phase(a, qcd::KIND_HB, 0, rep & 3, b, L->stream) == cudaSuccess &&
           L->ops->phase(a, qcd::KIND_OR, 1, rep & 3, b, L->stream) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e1, L->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = b;
    }
  }
  int rc = best ? QCD_OK : set_error(QCD_ERR_CUDA, "autotune: no launch shape worked");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, L->stream);
  cudaFreeAsync(dummy, L->stream);
  cudaError_t e = cudaStreamSynchronize(L->stream);
  if (rc != QCD_OK) return rc;
  if (e != cudaSuccess) return set_error(QCD_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  L->block = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  tune_store_locked();
  return QCD_OK;
}

}  // namespace

namespace qcd {
int set_last_error(int code, const char* msg) { return set_error(code, "%s", msg); }
}  // namespace qcd

extern "C" {

const char* qcd_last_error(void) { return g_last_error.c_str(); }

int qcd_lattice_create(qcd_lattice** out, int group, int Ns, int Nt, double beta, int flux, int precision,
                       int start, uint64_t seed, void* stream) {
  return qcd_lattice_create_ex(out, group, Ns, Nt, beta, flux, 0, QCD_FIELD_LINKS, precision, start, seed, stream);
}

namespace {
int create_lattice(qcd_lattice** out, int group, int Ns, int Nt, double beta, int flux, int flux8, int field_mode,
                   int precision, int start, uint64_t seed, void* stream, int nt_device);
}

int qcd_lattice_create_ex(qcd_lattice** out, int group, int Ns, int Nt, double beta, int flux, int flux8,
                          int field_mode, int precision, int start, uint64_t seed, void* stream) {
  return create_lattice(out, group, Ns, Nt, beta, flux, flux8, field_mode, precision, start, seed, stream, -1);
}

int qcd_lattice_create_split(qcd_lattice** out, int group, int Ns, int Nt, double beta, int flux, int flux8,
                             int field_mode, int precision, int start, uint64_t seed, void* stream, int nt_device) {
  if (!out) return set_error(QCD_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (nt_device < 0 || nt_device > Nt)
    return set_error(QCD_ERR_INVALID_ARG, "nt_device must be in [0, Nt], got %d", nt_device);
  return create_lattice(out, group, Ns, Nt, beta, flux, flux8, field_mode, precision, start, seed, stream,
                        nt_device);
}

int qcd_get_residency(qcd_lattice* L, size_t* device_bytes, size_t* host_bytes, int* nt_device) {
  if (int rc = check(L)) return rc;
  if (!device_bytes || !host_bytes || !nt_device) return set_error(QCD_ERR_INVALID_ARG, "null output pointer");
  const size_t n_arrays = size_t(L->ops->comps) * 8;
  const size_t array_bytes = L->link_bytes / n_arrays;
  const size_t dev = L->split ? L->split_device_bytes : array_bytes;
  *device_bytes = n_arrays * dev;
  *host_bytes = n_arrays * (array_bytes - dev);
  // t-slices wholly in device memory: each t-slice of an array is Ns^3/2 vectors of 16 bytes
  const size_t slice = size_t(L->Ns) * L->Ns * L->Ns / 2 * 16;
  *nt_device = int(std::min<size_t>(size_t(L->Nt), dev / slice));
  return QCD_OK;
}

namespace {
int create_lattice(qcd_lattice** out, int group, int Ns, int Nt, double beta, int flux, int flux8, int field_mode,
                   int precision, int start, uint64_t seed, void* stream, int nt_device) {
  if (!out) return set_error(QCD_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (group == 2 && flux8 != 0) return set_error(QCD_ERR_INVALID_ARG, "the lambda8 flux needs SU(3)");
  if (field_mode != QCD_FIELD_LINKS && field_mode != QCD_FIELD_FROZEN)
    return set_error(QCD_ERR_INVALID_ARG, "unknown field mode %d", field_mode);
  if (group != 2 && group != 3) return set_error(QCD_ERR_INVALID_ARG, "group must be 2 or 3, got %d", group);
  if (Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1))
    return set_error(QCD_ERR_INVALID_ARG, "Ns and Nt must be even and >= 2 (got %d, %d)", Ns, Nt);
  const long long V = (long long)Ns * Ns * Ns * Nt;
  if (V >= (1LL << 31) || Ns > 1290) return set_error(QCD_ERR_INVALID_ARG, "lattice too large (V = %lld)", V);
  if (!(beta >= 0.0)) return set_error(QCD_ERR_INVALID_ARG, "beta must be >= 0");
  if (precision != QCD_FP64_PLAIN && precision != QCD_FP32_COMPRESSED)
    return set_error(QCD_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (start != QCD_COLD && start != QCD_HOT) return set_error(QCD_ERR_INVALID_ARG, "unknown start %d", start);

  qcd_lattice* L = new (std::nothrow) qcd_lattice();
  if (!L) return set_error(QCD_ERR_OOM, "host allocation failed");
  L->ops = pick_ops(group, precision);
  L->group = group;
  L->precision = precision;
  L->Ns = Ns;
  L->Nt = Nt;
  L->flux = flux;
  L->flux8 = flux8;
  L->field_mode = field_mode;
  L->beta = beta;
  L->seed = seed;
  L->stream = static_cast<cudaStream_t>(stream);
  L->g.Ns = Ns;
  L->g.Nt = Nt;
  L->g.Vh = int(V / 2);
  qcd::geom_set_decode(L->g);
  L->g.plane = (L->g.Vh + 63) / 64 * 64;
  L->link_bytes = size_t(L->ops->comps) * 8 * size_t(L->g.plane) * 16;
  auto fail = [&](int rc) {
    qcd_lattice_destroy(L);
    return rc;
  };
  cudaError_t e = cudaGetDevice(&L->device);
  if (e != cudaSuccess) return fail(set_error(QCD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)));
  if (nt_device >= 0) {
    // Every link array padded to a whole number of mapping granules; its
    // first t-slices (rounded up to a granule) in device memory, the rest in
    // host memory.
    size_t gran = 0;
    const int node = qcd::split_host_node(L->device, &gran);
    if (node < 0)
      return fail(set_error(QCD_ERR_NOT_SUPPORTED, "this device cannot map host-NUMA memory into its address space"));
    const size_t vecs = gran / 16;
    L->g.plane = int64_t((size_t(L->g.Vh) + vecs - 1) / vecs * vecs);
    const size_t n_arrays = size_t(L->ops->comps) * 8, array_bytes = size_t(L->g.plane) * 16;
    L->link_bytes = n_arrays * array_bytes;
    const size_t want = size_t(nt_device) * (size_t(Ns) * Ns * Ns / 2) * 16;
    L->split_device_bytes = std::min(array_bytes, (want + gran - 1) / gran * gran);
    char why[256] = {0};
    if (int rc = qcd::split_alloc(L->device, node, gran, n_arrays, array_bytes, L->split_device_bytes, &L->split,
                                  &L->links, why, sizeof why))
      return fail(set_error(rc, "%s", why));
  } else if (cudaMalloc(&L->links, L->link_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_error(QCD_ERR_OOM, "device allocation of %zu bytes of links failed", L->link_bytes));
  }
  const size_t n_part = std::max(qcd::measure_partials(L->g), qcd::fused_partials(L->g));
  const size_t small_bytes = 256;
  if (cudaMalloc(reinterpret_cast<void**>(&L->d_small), small_bytes) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L->d_partials), n_part * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L->d_phase64), 4 * Ns * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L->d_phase32), 4 * Ns * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_error(QCD_ERR_OOM, "device allocation of %zu bytes of links failed", L->link_bytes));
  }
  L->d_sweep = reinterpret_cast<uint32_t*>(L->d_small);
  L->d_exhausted = reinterpret_cast<unsigned long long*>(L->d_small + 8);
  L->d_meas = reinterpret_cast<double*>(L->d_small + 64);
  if ((e = cudaMemsetAsync(L->d_small, 0, small_bytes, L->stream)) != cudaSuccess)
    return fail(set_error(QCD_ERR_CUDA, "memset: %s", cudaGetErrorString(e)));
  phase_table_kernel<<<(Ns + 63) / 64, 64, 0, L->stream>>>(L->d_phase64, L->d_phase32, Ns, flux, flux8);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(set_error(QCD_ERR_CUDA, "phase table: %s", cudaGetErrorString(e)));
  if ((e = L->ops->start(make_ctx(L, seed), start, L->stream)) != cudaSuccess)
    return fail(set_error(QCD_ERR_CUDA, "start: %s", cudaGetErrorString(e)));
  if (field_mode == QCD_FIELD_FROZEN && (e = L->ops->set_frozen(make_ctx(L, seed), L->stream)) != cudaSuccess)
    return fail(set_error(QCD_ERR_CUDA, "frozen links: %s", cudaGetErrorString(e)));
  if ((e = cudaStreamSynchronize(L->stream)) != cudaSuccess)
    return fail(set_error(QCD_ERR_CUDA, "create: %s", cudaGetErrorString(e)));
  *out = L;
  return QCD_OK;
}
}  // namespace

int qcd_get_field_mode(qcd_lattice* L, int* field_mode) {
  if (int rc = check(L)) return rc;
  if (!field_mode) return set_error(QCD_ERR_INVALID_ARG, "field_mode is null");
  *field_mode = L->field_mode;
  return QCD_OK;
}

int qcd_lattice_destroy(qcd_lattice* L) {
  if (!L) return QCD_OK;
  if (L->stream) cudaStreamSynchronize(L->stream);
  else cudaDeviceSynchronize();
  drop_graphs(L);
  for (cudaEvent_t e : L->meas_ev)
    if (e) cudaEventDestroy(e);
  if (L->split) qcd::split_free(L->split);
  else cudaFree(L->links);
  cudaFree(L->d_small);
  cudaFree(L->d_partials);
  cudaFree(L->d_phase64);
  cudaFree(L->d_phase32);
  delete L;
  return QCD_OK;
}

int qcd_set_nhit(qcd_lattice* L, int nhit) {
  if (int rc = check(L)) return rc;
  if (nhit < 1) return set_error(QCD_ERR_INVALID_ARG, "nhit must be >= 1");
  L->nhit = nhit;
  return QCD_OK;
}

int qcd_set_block(qcd_lattice* L, int threads) {
  if (int rc = check(L)) return rc;
  if (threads != 0 && (threads < 32 || threads > 1024 || threads % 32))
    return set_error(QCD_ERR_INVALID_ARG, "threads must be 0 or a multiple of 32 in [32, 1024]");
  if (threads > L->ops->max_phase_block())
    return set_error(QCD_ERR_INVALID_ARG, "the phase kernels launch with at most %d threads per block",
                     L->ops->max_phase_block());
  L->block = threads;
  return QCD_OK;
}

int qcd_get_block(const qcd_lattice* L, int* threads) {
  if (int rc = check(L)) return rc;
  if (!threads) return set_error(QCD_ERR_INVALID_ARG, "threads is null");
  *threads = L->block;
  return QCD_OK;
}

int qcd_sweep(qcd_lattice* L, int n_heatbath, int n_overrelax, uint64_t seed) {
  if (int rc = check(L)) return rc;
  if (n_heatbath < 0 || n_overrelax < 0) return set_error(QCD_ERR_INVALID_ARG, "negative pass count");
  if (n_heatbath == 0) return QCD_OK;
  if (int rc = use_device(L)) return rc;
  if (L->block == 0)
    if (int rc = autotune(L)) return rc;
  SweepGraph* g = nullptr;
  if (int rc = get_graph(L, seed, n_overrelax, false, &g)) return rc;
  for (int i = 0; i < n_heatbath; ++i) {
    if (i > 0 && L->profiling)
      if (int rc = get_graph(L, seed, n_overrelax, false, &g)) return rc;  // the other instance
    if (int rc = launch_graph(L, *g)) return rc;
  }
  return QCD_OK;
}

// Block size of phases launched one at a time (qcd_phase) and of the fused
// measurement's final sums that follow them.
static int phase_block(const qcd_lattice* L) { return L->block ? L->block : 128; }

static bool fused_measure_available(const qcd_lattice* L) {
  return L->ops->measure_fused_tail != nullptr && L->field_mode == QCD_FIELD_LINKS;
}

static int measure_impl(qcd_lattice* L, int effective, double* plaq, double* poly);

int qcd_working_sweep(qcd_lattice* L, int n_heatbath, int n_overrelax, uint64_t seed, double* host_out, int wait) {
  if (int rc = check(L)) return rc;
  if (n_heatbath < 1 || n_overrelax < 0) return set_error(QCD_ERR_INVALID_ARG, "need n_heatbath >= 1, n_overrelax >= 0");
  if (!host_out) return set_error(QCD_ERR_INVALID_ARG, "host_out is null");
  if (int rc = use_device(L)) return rc;
  const bool fused = fused_measure_available(L) && n_overrelax > 0;
  if (!fused) {  // separate measurement after the sweeps
    if (int rc = qcd_sweep(L, n_heatbath, n_overrelax, seed)) return rc;
    if (wait) return measure_impl(L, 1, host_out, host_out + 3);
    QCD_CUDA(L->ops->measure(make_ctx(L, L->seed), 1, L->stream));
    QCD_CUDA(cudaMemcpyAsync(host_out, L->d_meas, 5 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    return QCD_OK;
  }
  if (n_heatbath > 1)
    if (int rc = qcd_sweep(L, n_heatbath - 1, n_overrelax, seed)) return rc;
  if (L->block == 0)
    if (int rc = autotune(L)) return rc;
  SweepGraph* g = nullptr;
  if (int rc = get_graph(L, seed, n_overrelax, true, &g)) return rc;
  if (int rc = launch_graph(L, *g)) return rc;
  QCD_CUDA(cudaMemcpyAsync(host_out, L->d_meas, 5 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  if (wait) QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

int qcd_phase(qcd_lattice* L, int kind, int parity, int mu, uint64_t seed) {
  if (int rc = check(L)) return rc;
  if (kind < QCD_HEATBATH || kind > QCD_OVERRELAX_MEASURE || (parity & ~1) || mu < 0 || mu > 3)
    return set_error(QCD_ERR_INVALID_ARG, "bad phase (kind %d, parity %d, mu %d)", kind, parity, mu);
  if (kind == QCD_OVERRELAX_MEASURE) {
    if (parity != 1 || mu < 1)
      return set_error(QCD_ERR_INVALID_ARG,
                       "QCD_OVERRELAX_MEASURE is a phase of odd parity with mu >= 1 (got parity %d, mu %d)",
                       parity, mu);
    if (!fused_measure_available(L))
      return set_error(QCD_ERR_NOT_SUPPORTED,
                       "the fused measurement needs FP32 SU(3) or SU(2) storage and the effective-link field mode");
  }
  if (int rc = use_device(L)) return rc;
  static const int kinds[4] = {qcd::KIND_HB, qcd::KIND_OR, qcd::KIND_OR_REUNIT, qcd::KIND_OR_MEAS};
  QCD_CUDA(L->ops->phase(make_ctx(L, seed), kinds[kind], parity, mu, phase_block(L), L->stream));
  return QCD_OK;
}

int qcd_measure_fused_finish(qcd_lattice* L, double* host_out) {
  if (int rc = check(L)) return rc;
  if (!host_out) return set_error(QCD_ERR_INVALID_ARG, "host_out is null");
  if (!fused_measure_available(L))
    return set_error(QCD_ERR_NOT_SUPPORTED,
                     "the fused measurement needs FP32 SU(3) or SU(2) storage and the effective-link field mode");
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(L->ops->measure_fused_tail(make_ctx(L, L->seed), phase_block(L), L->stream));
  QCD_CUDA(cudaMemcpyAsync(host_out, L->d_meas, 8 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

int qcd_reunitarize(qcd_lattice* L) {
  if (int rc = check(L)) return rc;
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(L->ops->reunit(make_ctx(L, L->seed), 0, L->stream));
  return QCD_OK;
}

static int measure_impl(qcd_lattice* L, int effective, double* plaq, double* poly) {
  if (int rc = check(L)) return rc;
  if (int rc = use_device(L)) return rc;
  if (L->profiling) QCD_CUDA(cudaEventRecord(L->meas_ev[0], L->stream));
  QCD_CUDA(L->ops->measure(make_ctx(L, L->seed), effective, L->stream));
  if (L->profiling) QCD_CUDA(cudaEventRecord(L->meas_ev[1], L->stream));
  double h[5];
  QCD_CUDA(cudaMemcpyAsync(h, L->d_meas, sizeof h, cudaMemcpyDeviceToHost, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  if (L->profiling) {
    float ms = 0.f;
    QCD_CUDA(cudaEventElapsedTime(&ms, L->meas_ev[0], L->meas_ev[1]));
    L->prof_ms[QCD_PROF_MEASURE] += ms;
    L->prof_launches[QCD_PROF_MEASURE] += 2;
  }
  if (plaq) {
    plaq[0] = h[0];
    plaq[1] = h[1];
    plaq[2] = h[2];
  }
  if (poly) {
    poly[0] = h[3];
    poly[1] = h[4];
  }
  return QCD_OK;
}

int qcd_measure(qcd_lattice* L, double* plaquette, double* polyakov) {
  return measure_impl(L, 1, plaquette, polyakov);
}

int qcd_measure_async(qcd_lattice* L, double* host_out) {
  if (int rc = check(L)) return rc;
  if (!host_out) return set_error(QCD_ERR_INVALID_ARG, "host_out is null");
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(L->ops->measure(make_ctx(L, L->seed), 1, L->stream));
  QCD_CUDA(cudaMemcpyAsync(host_out, L->d_meas, 5 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  return QCD_OK;
}

int qcd_measure_bare(qcd_lattice* L, double* plaquette) { return measure_impl(L, 0, plaquette, nullptr); }

static size_t canonical_bytes(const qcd_lattice* L) {
  return size_t(2) * L->g.Vh * 4 * L->group * L->group * 2 * sizeof(double);
}

int qcd_get_links(qcd_lattice* L, double* host_out) {
  if (int rc = check(L)) return rc;
  if (!host_out) return set_error(QCD_ERR_INVALID_ARG, "host_out is null");
  if (int rc = use_device(L)) return rc;
  double* tmp = nullptr;
  const size_t bytes = canonical_bytes(L);
  if (cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, L->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_error(QCD_ERR_OOM, "temporary of %zu bytes", bytes);
  }
  cudaError_t e = L->ops->to_canonical(make_ctx(L, L->seed), tmp, L->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, bytes, cudaMemcpyDeviceToHost, L->stream);
  cudaFreeAsync(tmp, L->stream);
  cudaError_t e2 = cudaStreamSynchronize(L->stream);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return set_error(QCD_ERR_CUDA, "get_links: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return QCD_OK;
}

int qcd_set_links(qcd_lattice* L, const double* host_in) {
  if (int rc = check(L)) return rc;
  if (!host_in) return set_error(QCD_ERR_INVALID_ARG, "host_in is null");
  if (int rc = use_device(L)) return rc;
  double* tmp = nullptr;
  const size_t bytes = canonical_bytes(L);
  if (cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, L->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_error(QCD_ERR_OOM, "temporary of %zu bytes", bytes);
  }
  cudaError_t e = cudaMemcpyAsync(tmp, host_in, bytes, cudaMemcpyHostToDevice, L->stream);
  if (e == cudaSuccess) e = L->ops->from_canonical(make_ctx(L, L->seed), tmp, L->stream);
  cudaFreeAsync(tmp, L->stream);
  cudaError_t e2 = cudaStreamSynchronize(L->stream);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return set_error(QCD_ERR_CUDA, "set_links: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return QCD_OK;
}

int qcd_link_bytes(const qcd_lattice* L, size_t* bytes) {
  if (int rc = check(L)) return rc;
  if (!bytes) return set_error(QCD_ERR_INVALID_ARG, "bytes is null");
  *bytes = L->link_bytes;
  return QCD_OK;
}

int qcd_copy_links_in(qcd_lattice* L, const void* host_in, size_t bytes) {
  if (int rc = check(L)) return rc;
  if (!host_in || bytes != L->link_bytes)
    return set_error(QCD_ERR_INVALID_ARG, "need %zu bytes of raw storage", L->link_bytes);
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaMemcpyAsync(L->links, host_in, bytes, cudaMemcpyHostToDevice, L->stream));
  return QCD_OK;
}

int qcd_copy_links_out(qcd_lattice* L, void* host_out, size_t bytes) {
  if (int rc = check(L)) return rc;
  if (!host_out || bytes != L->link_bytes)
    return set_error(QCD_ERR_INVALID_ARG, "need %zu bytes of raw storage", L->link_bytes);
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaMemcpyAsync(host_out, L->links, bytes, cudaMemcpyDeviceToHost, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

int qcd_get_sweep(qcd_lattice* L, uint32_t* sweep) {
  if (int rc = check(L)) return rc;
  if (!sweep) return set_error(QCD_ERR_INVALID_ARG, "sweep is null");
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaMemcpyAsync(sweep, L->d_sweep, sizeof(uint32_t), cudaMemcpyDeviceToHost, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

int qcd_set_sweep(qcd_lattice* L, uint32_t sweep) {
  if (int rc = check(L)) return rc;
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaMemcpyAsync(L->d_sweep, &sweep, sizeof(uint32_t), cudaMemcpyHostToDevice, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

int qcd_set_profiling(qcd_lattice* L, int enable) {
  if (int rc = check(L)) return rc;
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(L->stream ? cudaStreamSynchronize(L->stream) : cudaDeviceSynchronize());
  for (auto& e : L->meas_ev)
    if (!e) QCD_CUDA(cudaEventCreate(&e));
  for (auto& g : L->graphs) g.pending = false;  // totals restart
  L->profiling = enable ? 1 : 0;
  for (int k = 0; k < QCD_PROF_N; ++k) {
    L->prof_ms[k] = 0.0;
    L->prof_launches[k] = 0;
  }
  return QCD_OK;
}

int qcd_get_profile(qcd_lattice* L, double* ms, unsigned long long* launches) {
  if (int rc = check(L)) return rc;
  if (!ms || !launches) return set_error(QCD_ERR_INVALID_ARG, "null output");
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  if (int rc = fold_all(L)) return rc;
  for (int k = 0; k < QCD_PROF_N; ++k) {
    ms[k] = L->prof_ms[k];
    launches[k] = L->prof_launches[k];
  }
  return QCD_OK;
}

namespace {
struct CheckpointHeader {
  char magic[8];
  uint32_t version, group, precision, Ns, Nt;
  int32_t flux;
  uint32_t nhit, lattice_id, sweep, field_mode;  // field_mode 0 in files written before the mode existed
  uint64_t seed;
  double beta;
  uint64_t exhausted;
};
static_assert(sizeof(CheckpointHeader) == 72, "checkpoint header layout");
constexpr char kMagic[8] = {'Q', 'C', 'D', 'G', 'B', '3', '0', '0'};
}  // namespace

int qcd_save(qcd_lattice* L, const char* path) {
  if (int rc = check(L)) return rc;
  if (!path) return set_error(QCD_ERR_INVALID_ARG, "path is null");
  CheckpointHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.group = uint32_t(L->group);
  h.precision = uint32_t(L->precision);
  h.Ns = uint32_t(L->Ns);
  h.Nt = uint32_t(L->Nt);
  h.flux = L->flux;
  h.field_mode = uint32_t(L->field_mode);
  h.nhit = uint32_t(L->nhit);
  h.lattice_id = L->lattice_id;
  h.seed = L->seed;
  h.beta = L->beta;
  if (int rc = qcd_get_sweep(L, &h.sweep)) return rc;
  unsigned long long ex = 0;
  if (int rc = qcd_get_exhausted(L, &ex)) return rc;
  h.exhausted = ex;
  const size_t n = canonical_bytes(L) / sizeof(double);
  std::vector<double> buf(n);
  if (int rc = qcd_get_links(L, buf.data())) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(QCD_ERR_INVALID_ARG, "cannot open %s for writing", path);
  // the 8 bytes after the header: lambda8 flux (int32; 0 in files written
  // before it existed) and 4 reserved zero bytes
  const int32_t tail[2] = {int32_t(L->flux8), 0};
  const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(tail, 8, 1, f) == 1 &&
                  fwrite(buf.data(), sizeof(double), n, f) == n;
  if (fclose(f) != 0 || !ok) return set_error(QCD_ERR_INVALID_ARG, "writing %s failed", path);
  return QCD_OK;
}

int qcd_lattice_load(qcd_lattice** out, const char* path, int precision, void* stream) {
  if (!out || !path) return set_error(QCD_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(QCD_ERR_INVALID_ARG, "cannot open %s", path);
  CheckpointHeader h{};
  int32_t tail[2] = {0, 0};
  if (fread(&h, sizeof h, 1, f) != 1 || fread(tail, 8, 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 ||
      h.version != 1 || (h.group != 2 && h.group != 3) || h.field_mode > 1 || h.Ns < 2 || h.Nt < 2 || h.Ns > 1290 || h.Nt > (1u << 30)) {
    fclose(f);
    return set_error(QCD_ERR_INVALID_ARG, "%s is not a version-1 checkpoint", path);
  }
  qcd_lattice* L = nullptr;
  int rc = qcd_lattice_create_ex(&L, int(h.group), int(h.Ns), int(h.Nt), h.beta, h.flux, int(tail[0]),
                                 int(h.field_mode),
                                 precision, QCD_COLD, h.seed, stream);
  if (rc) {
    fclose(f);
    return rc;
  }
  const size_t n = canonical_bytes(L) / sizeof(double);
  std::vector<double> buf(n);
  const bool ok = fread(buf.data(), sizeof(double), n, f) == n;
  fclose(f);
  if (!ok) {
    qcd_lattice_destroy(L);
    return set_error(QCD_ERR_INVALID_ARG, "%s is truncated", path);
  }
  L->nhit = int(h.nhit);
  L->lattice_id = h.lattice_id;
  if ((rc = qcd_set_links(L, buf.data())) || (rc = qcd_set_sweep(L, h.sweep))) {
    qcd_lattice_destroy(L);
    return rc;
  }
  const unsigned long long ex = h.exhausted;
  cudaError_t e = cudaMemcpyAsync(L->d_exhausted, &ex, sizeof ex, cudaMemcpyHostToDevice, L->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  if (e != cudaSuccess) {
    qcd_lattice_destroy(L);
    return set_error(QCD_ERR_CUDA, "load: %s", cudaGetErrorString(e));
  }
  *out = L;
  return QCD_OK;
}

int qcd_get_exhausted(qcd_lattice* L, unsigned long long* count) {
  if (int rc = check(L)) return rc;
  if (!count) return set_error(QCD_ERR_INVALID_ARG, "count is null");
  if (int rc = use_device(L)) return rc;
  QCD_CUDA(cudaMemcpyAsync(count, L->d_exhausted, sizeof(unsigned long long), cudaMemcpyDeviceToHost, L->stream));
  QCD_CUDA(cudaStreamSynchronize(L->stream));
  return QCD_OK;
}

}  // extern "C"
