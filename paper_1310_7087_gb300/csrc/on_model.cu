// on_model.cu -- the O(N) model sweep (N-component real scalar field on the
// sites, lattice phi^4 action) by multi-hit Metropolis, and its C ABI.
//
// Action:  S = sum_x [ -2 kappa sum_mu phi_x.phi_{x+mu} + phi_x.phi_x
//                      + lambda (phi_x.phi_x - 1)^2 ].
// A checkerboard phase visits every site of one parity; a visit makes nhit
// Metropolis hits with the eight neighbours fixed: hit h proposes
// phi' = phi + delta (2u - 1) componentwise (Philox block (s, sweep, 3 << 4, h))
// and accepts iff dS <= 0 or u < exp(-dS), u = word h mod 4 of block
// (s, sweep, 4 << 4, h / 4).  The local action of a value needs only
// F = sum of the neighbours: s(phi) = -2 kappa phi.F + phi.phi
// + lambda (phi.phi - 1)^2.
//
// Storage: one 16-byte vector per site and parity (FP32: float4; FP64: two
// double2 planes), even/odd halves, components beyond N kept zero.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "qcd.h"
#include "qcd_device.cuh"

namespace qcd {
namespace {

enum : uint32_t { KIND_ON_START = 2u, KIND_ON_PROPOSE = 3u, KIND_ON_ACCEPT = 4u };

constexpr int ON_MEAS_THREADS = 256;
constexpr int ON_MEAS_VALUES = 6;  // phi.phi, hopping term, M_0..M_3

struct OnCtx {
  void* phi;
  GeomH g;
  int N;
  int nhit;
  double kappa, lambda, delta;
  uint32_t k0, k1;
  const uint32_t* sweep;
  uint32_t* sweep_rw;
  unsigned long long* accepted;
  double* partials;
  double* meas_out;
};

template <typename R>
struct OnStore;

template <>
struct OnStore<float> {
  static __device__ __forceinline__ void load(const OnCtx& a, int par, int h, float v[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a.phi) + par * a.g.plane + h);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
  static __device__ __forceinline__ void store(const OnCtx& a, int par, int h, const float v[4]) {
    reinterpret_cast<float4*>(a.phi)[par * a.g.plane + h] = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <>
struct OnStore<double> {
  static __device__ __forceinline__ void load(const OnCtx& a, int par, int h, double v[4]) {
    const double2* p = reinterpret_cast<const double2*>(a.phi);
    const double2 x = __ldg(p + par * a.g.plane + h);
    const double2 y = __ldg(p + (2 + par) * a.g.plane + h);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
  }
  static __device__ __forceinline__ void store(const OnCtx& a, int par, int h, const double v[4]) {
    double2* p = reinterpret_cast<double2*>(a.phi);
    p[par * a.g.plane + h] = make_double2(v[0], v[1]);
    p[(2 + par) * a.g.plane + h] = make_double2(v[2], v[3]);
  }
};

// The Metropolis test's exponential: FP32 from the hardware approximation
// (relative error ~2^-21, so a decision can only differ from an exact one when
// u lies within ~1e-6 of exp(-dS)); FP64 from the library.
__device__ __forceinline__ float q_exp(float x) { return __expf(x); }
__device__ __forceinline__ double q_exp(double x) { return exp(x); }

// s(phi) = -2 kappa phi.F + phi.phi + lambda (phi.phi - 1)^2
template <typename R, int N>
__device__ __forceinline__ R local_action(const R phi[4], const R F[4], R two_kappa, R lambda) {
  R pf = R(0), pp = R(0);
#pragma unroll
  for (int c = 0; c < N; ++c) {
    pf = fma(phi[c], F[c], pf);
    pp = fma(phi[c], phi[c], pp);
  }
  const R d = pp - R(1);
  return fma(-two_kappa, pf, fma(lambda * d, d, pp));
}

template <typename R, int D>
__device__ __forceinline__ void add_neighbours(const OnCtx& a, int par, const LexSite& x, R F[4]) {
  R v[4];
  const LexSite p = lex_step<D, +1>(a.g, x), m = lex_step<D, -1>(a.g, x);
  OnStore<R>::load(a, par, p.s >> 1, v);
#pragma unroll
  for (int c = 0; c < 4; ++c) F[c] += v[c];
  OnStore<R>::load(a, par, m.s >> 1, v);
#pragma unroll
  for (int c = 0; c < 4; ++c) F[c] += v[c];
}

template <typename R, int N>
__global__ void on_phase_kernel(const OnCtx a, int parity) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned n_acc = 0;
  if (h < a.g.Vh) {
    const Site sc = site_of(a.g, parity, h);
    LexSite x;
    x.c[0] = sc.x;
    x.c[1] = sc.y;
    x.c[2] = sc.z;
    x.c[3] = sc.t;
    x.s = 2 * h + (sc.x & 1);
    R F[4] = {R(0), R(0), R(0), R(0)};
    add_neighbours<R, 0>(a, parity ^ 1, x, F);
    add_neighbours<R, 1>(a, parity ^ 1, x, F);
    add_neighbours<R, 2>(a, parity ^ 1, x, F);
    add_neighbours<R, 3>(a, parity ^ 1, x, F);
    R phi[4];
    OnStore<R>::load(a, parity, h, phi);
    const R two_kappa = R(2.0 * a.kappa), lambda = R(a.lambda), delta = R(a.delta);
    R cur = local_action<R, N>(phi, F, two_kappa, lambda);
    const uint32_t sweep = *a.sweep;
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (int hit = 0; hit < a.nhit; ++hit) {
      const uint4 w = philox4x32_10(make_uint4(uint32_t(x.s), sweep, KIND_ON_PROPOSE << 4, uint32_t(hit)), a.k0, a.k1);
      if ((hit & 3) == 0)
        acc = philox4x32_10(make_uint4(uint32_t(x.s), sweep, KIND_ON_ACCEPT << 4, uint32_t(hit >> 2)), a.k0, a.k1);
      const uint32_t wu[4] = {w.x, w.y, w.z, w.w};
      R trial[4] = {phi[0], phi[1], phi[2], phi[3]};
#pragma unroll
      for (int c = 0; c < N; ++c) trial[c] = fma(delta, fma(R(2), u01<R>(wu[c]), R(-1)), phi[c]);
      const R next = local_action<R, N>(trial, F, two_kappa, lambda);
      const R dS = next - cur;
      const uint32_t aw = (hit & 3) == 0 ? acc.x : (hit & 3) == 1 ? acc.y : (hit & 3) == 2 ? acc.z : acc.w;
      if (dS <= R(0) || u01<R>(aw) < q_exp(-dS)) {
#pragma unroll
        for (int c = 0; c < N; ++c) phi[c] = trial[c];
        cur = next;
        ++n_acc;
      }
    }
    OnStore<R>::store(a, parity, h, phi);
  }
  // one atomic per warp for the acceptance count
  const unsigned total = __reduce_add_sync(0xffffffffu, n_acc);
  if ((threadIdx.x & 31) == 0 && total) atomicAdd(a.accepted, (unsigned long long)total);
}

__global__ void on_advance_kernel(const OnCtx a) { *a.sweep_rw += 1u; }

template <typename R>
__global__ void on_start_kernel(const OnCtx a, int hot) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 2LL * a.g.Vh) return;
  const int par = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  const Site x = site_of(a.g, par, h);
  const uint32_t s = uint32_t(lex(a.g, x));
  R v[4] = {R(0), R(0), R(0), R(0)};
  if (hot) {
    const uint4 w = philox4x32_10(make_uint4(s, 0xFFFFFFFFu, KIND_ON_START << 4, 0u), a.k0, a.k1);
    const uint32_t wu[4] = {w.x, w.y, w.z, w.w};
    for (int c = 0; c < a.N; ++c) v[c] = R(2.0 * u01<double>(wu[c]) - 1.0);
  } else {
    v[0] = R(1);
  }
  OnStore<R>::store(a, par, h, v);
}

// Canonical host order [s][c] (N doubles per site) <-> device layout.
template <typename R>
__global__ void on_to_canonical(const OnCtx a, double* out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 2LL * a.g.Vh) return;
  const int par = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  const int64_t s = lex(a.g, site_of(a.g, par, h));
  R v[4];
  OnStore<R>::load(a, par, h, v);
  for (int c = 0; c < a.N; ++c) out[s * a.N + c] = double(v[c]);
}

template <typename R>
__global__ void on_from_canonical(const OnCtx a, const double* in) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= 2LL * a.g.Vh) return;
  const int par = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
  const int64_t s = lex(a.g, site_of(a.g, par, h));
  R v[4] = {R(0), R(0), R(0), R(0)};
  for (int c = 0; c < a.N; ++c) v[c] = R(in[s * a.N + c]);
  OnStore<R>::store(a, par, h, v);
}

// Per-site phi.phi, forward hopping term sum_mu phi_x.phi_{x+mu}, and phi_x,
// in the storage precision per site and FP64 across sites: per-block partials
// in a fixed order, then one block sums the partials in a fixed order.
template <typename R>
__global__ void __launch_bounds__(ON_MEAS_THREADS) on_measure_kernel(const OnCtx a) {
  const int64_t idx = int64_t(blockIdx.x) * ON_MEAS_THREADS + threadIdx.x;
  double v[ON_MEAS_VALUES] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (idx < 2LL * a.g.Vh) {
    const int par = int(idx / a.g.Vh), h = int(idx % a.g.Vh);
    const Site x = site_of(a.g, par, h);
    R p[4];
    OnStore<R>::load(a, par, h, p);
    R pp = R(0), hop = R(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) pp = fma(p[c], p[c], pp);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const Site y = step(a.g, x, mu, +1);
      R q[4];
      OnStore<R>::load(a, par ^ 1, lex(a.g, y) >> 1, q);
#pragma unroll
      for (int c = 0; c < 4; ++c) hop = fma(p[c], q[c], hop);
    }
    v[0] = double(pp);
    v[1] = double(hop);
#pragma unroll
    for (int c = 0; c < 4; ++c) v[2 + c] = double(p[c]);
  }
  __shared__ double sh[ON_MEAS_VALUES][ON_MEAS_THREADS];
#pragma unroll
  for (int k = 0; k < ON_MEAS_VALUES; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = ON_MEAS_THREADS / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
#pragma unroll
      for (int k = 0; k < ON_MEAS_VALUES; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < ON_MEAS_VALUES) a.partials[ON_MEAS_VALUES * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(1024) on_measure_final(const OnCtx a, int n_blocks) {
  __shared__ double sh[ON_MEAS_VALUES][1024];
  double s[ON_MEAS_VALUES] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_blocks; b += 1024)
#pragma unroll
    for (int k = 0; k < ON_MEAS_VALUES; ++k) s[k] += a.partials[ON_MEAS_VALUES * b + k];
#pragma unroll
  for (int k = 0; k < ON_MEAS_VALUES; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w)
#pragma unroll
      for (int k = 0; k < ON_MEAS_VALUES; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double V = 2.0 * double(a.g.Vh);
    a.meas_out[0] = sh[0][0] / V;
    a.meas_out[1] = sh[1][0] / (4.0 * V);
    double m2 = 0.0;
    for (int c = 0; c < 4; ++c) {
      const double m = sh[2 + c][0] / V;
      a.meas_out[3 + c] = m;
      m2 += m * m;
    }
    a.meas_out[2] = sqrt(m2);
  }
}

template <typename R>
cudaError_t launch_on_phase(const OnCtx& a, int parity, int block, cudaStream_t st) {
  const unsigned grid = unsigned((a.g.Vh + block - 1) / block);
  switch (a.N) {
    case 1: on_phase_kernel<R, 1><<<grid, block, 0, st>>>(a, parity); break;
    case 2: on_phase_kernel<R, 2><<<grid, block, 0, st>>>(a, parity); break;
    case 3: on_phase_kernel<R, 3><<<grid, block, 0, st>>>(a, parity); break;
    default: on_phase_kernel<R, 4><<<grid, block, 0, st>>>(a, parity); break;
  }
  return cudaGetLastError();
}

thread_local char g_msg[512];

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return set_last_error(code, g_msg);
}

}  // namespace
}  // namespace qcd

using namespace qcd;

struct qcd_on {
  int N = 0, Ns = 0, Nt = 0, precision = 0, nhit = 100, block = 128;
  double kappa = 0.0, lambda = 0.0, delta = 1.0;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  GeomH g{};
  void* phi = nullptr;
  unsigned char* d_small = nullptr;  // sweep counter, accepted hits, results
  double* d_partials = nullptr;
  int n_meas_blocks = 0;
  cudaGraphExec_t graph = nullptr;  // one sweep, for (graph_seed, nhit, block)
  uint64_t graph_seed = 0;
  int graph_nhit = 0, graph_block = 0;
};

namespace {

OnCtx make_on_ctx(const qcd_on* L, uint64_t seed) {
  OnCtx a{};
  a.phi = L->phi;
  a.g = L->g;
  a.N = L->N;
  a.nhit = L->nhit;
  a.kappa = L->kappa;
  a.lambda = L->lambda;
  a.delta = L->delta;
  a.k0 = uint32_t(seed);  // lattice id 0
  a.k1 = uint32_t(seed >> 32);
  a.sweep = reinterpret_cast<const uint32_t*>(L->d_small);
  a.sweep_rw = reinterpret_cast<uint32_t*>(L->d_small);
  a.accepted = reinterpret_cast<unsigned long long*>(L->d_small + 8);
  a.partials = L->d_partials;
  a.meas_out = reinterpret_cast<double*>(L->d_small + 64);
  return a;
}

cudaError_t on_phase_launch(const qcd_on* L, int parity, uint64_t seed) {
  const OnCtx a = make_on_ctx(L, seed);
  return L->precision == QCD_FP64_PLAIN ? launch_on_phase<double>(a, parity, L->block, L->stream)
                                        : launch_on_phase<float>(a, parity, L->block, L->stream);
}

int check(const qcd_on* L) { return L ? QCD_OK : fail(QCD_ERR_INVALID_ARG, "null O(N) handle"); }

void drop_graph(qcd_on* L) {
  if (L->graph) cudaGraphExecDestroy(L->graph);
  L->graph = nullptr;
}

int build_graph(qcd_on* L, uint64_t seed) {
  drop_graph(L);
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
    return fail(QCD_ERR_CUDA, "O(N) graph: stream creation failed");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    qcd_on tmp = *L;
    tmp.stream = cap;
    const OnCtx a = make_on_ctx(&tmp, seed);
    cudaError_t e1 = on_phase_launch(&tmp, 0, seed);
    cudaError_t e2 = on_phase_launch(&tmp, 1, seed);
    on_advance_kernel<<<1, 1, 0, cap>>>(a);
    cudaError_t e3 = cudaGetLastError();
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&L->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    L->graph = nullptr;
    cudaGetLastError();
    return fail(QCD_ERR_CUDA, "O(N) graph: %s", cudaGetErrorString(e));
  }
  L->graph_seed = seed;
  L->graph_nhit = L->nhit;
  L->graph_block = L->block;
  return QCD_OK;
}

template <typename F>
int copy_via_device(qcd_on* L, size_t bytes, F&& body) {
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), bytes, L->stream);
  if (e != cudaSuccess) return fail(QCD_ERR_OOM, "O(N): %zu bytes of staging: %s", bytes, cudaGetErrorString(e));
  e = body(d);
  cudaFreeAsync(d, L->stream);
  const cudaError_t e2 = cudaStreamSynchronize(L->stream);
  if (e == cudaSuccess) e = e2;
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) field copy: %s", cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int qcd_on_create(qcd_on** out, int N, int Ns, int Nt, double kappa, double lambda, double delta, int precision,
                  int start, uint64_t seed, void* stream) {
  if (!out) return fail(QCD_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (N < 1 || N > 4) return fail(QCD_ERR_INVALID_ARG, "N must be 1..4, got %d", N);
  if (Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1))
    return fail(QCD_ERR_INVALID_ARG, "Ns and Nt must be even and >= 2 (got %d, %d)", Ns, Nt);
  const long long V = (long long)Ns * Ns * Ns * Nt;
  if (V >= (1LL << 31) || Ns > 1290) return fail(QCD_ERR_INVALID_ARG, "lattice too large (V = %lld)", V);
  if (!(delta > 0.0) || !(kappa == kappa) || !(lambda == lambda))
    return fail(QCD_ERR_INVALID_ARG, "delta must be > 0 and kappa, lambda finite");
  if (precision != QCD_FP64_PLAIN && precision != QCD_FP32_COMPRESSED)
    return fail(QCD_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (start != QCD_COLD && start != QCD_HOT) return fail(QCD_ERR_INVALID_ARG, "unknown start %d", start);
  qcd_on* L = new (std::nothrow) qcd_on();
  if (!L) return fail(QCD_ERR_OOM, "host allocation failed");
  L->N = N;
  L->Ns = Ns;
  L->Nt = Nt;
  L->precision = precision;
  L->kappa = kappa;
  L->lambda = lambda;
  L->delta = delta;
  L->seed = seed;
  L->stream = static_cast<cudaStream_t>(stream);
  L->g.Ns = Ns;
  L->g.Nt = Nt;
  L->g.Vh = int(V / 2);
  geom_set_decode(L->g);
  L->g.plane = (L->g.Vh + 63) / 64 * 64;
  L->n_meas_blocks = int((V + ON_MEAS_THREADS - 1) / ON_MEAS_THREADS);
  const size_t field_bytes = size_t(2) * size_t(L->g.plane) * 16 * (precision == QCD_FP64_PLAIN ? 2 : 1);
  if (cudaMalloc(&L->phi, field_bytes) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L->d_small), 256) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L->d_partials), sizeof(double) * ON_MEAS_VALUES * L->n_meas_blocks) !=
          cudaSuccess) {
    cudaGetLastError();
    qcd_on_destroy(L);
    return fail(QCD_ERR_OOM, "device allocation of %zu bytes of field failed", field_bytes);
  }
  cudaError_t e = cudaMemsetAsync(L->d_small, 0, 256, L->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(L->phi, 0, field_bytes, L->stream);
  if (e == cudaSuccess) {
    const OnCtx a = make_on_ctx(L, seed);
    const unsigned grid = unsigned((V + 255) / 256);
    if (precision == QCD_FP64_PLAIN) on_start_kernel<double><<<grid, 256, 0, L->stream>>>(a, start);
    else on_start_kernel<float><<<grid, 256, 0, L->stream>>>(a, start);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  if (e != cudaSuccess) {
    qcd_on_destroy(L);
    return fail(QCD_ERR_CUDA, "O(N) create: %s", cudaGetErrorString(e));
  }
  *out = L;
  return QCD_OK;
}

int qcd_on_destroy(qcd_on* L) {
  if (!L) return QCD_OK;
  if (L->stream) cudaStreamSynchronize(L->stream);
  else cudaDeviceSynchronize();
  drop_graph(L);
  cudaFree(L->phi);
  cudaFree(L->d_small);
  cudaFree(L->d_partials);
  delete L;
  return QCD_OK;
}

int qcd_on_set_nhit(qcd_on* L, int nhit) {
  if (int rc = check(L)) return rc;
  if (nhit < 1) return fail(QCD_ERR_INVALID_ARG, "nhit must be >= 1");
  L->nhit = nhit;
  return QCD_OK;
}

int qcd_on_set_block(qcd_on* L, int threads) {
  if (int rc = check(L)) return rc;
  if (threads != 64 && threads != 128 && threads != 256 && threads != 512)
    return fail(QCD_ERR_INVALID_ARG, "threads must be 64, 128, 256 or 512");
  L->block = threads;
  return QCD_OK;
}

int qcd_on_sweep(qcd_on* L, int n_sweeps, uint64_t seed) {
  if (int rc = check(L)) return rc;
  if (n_sweeps < 0) return fail(QCD_ERR_INVALID_ARG, "n_sweeps must be >= 0");
  if (n_sweeps == 0) return QCD_OK;
  if (!L->graph || L->graph_seed != seed || L->graph_nhit != L->nhit || L->graph_block != L->block)
    if (int rc = build_graph(L, seed)) return rc;
  for (int i = 0; i < n_sweeps; ++i) {
    const cudaError_t e = cudaGraphLaunch(L->graph, L->stream);
    if (e != cudaSuccess) return fail(QCD_ERR_CUDA, "O(N) sweep: %s", cudaGetErrorString(e));
  }
  return QCD_OK;
}

int qcd_on_phase(qcd_on* L, int parity, uint64_t seed) {
  if (int rc = check(L)) return rc;
  if (parity != 0 && parity != 1) return fail(QCD_ERR_INVALID_ARG, "parity must be 0 or 1");
  const cudaError_t e = on_phase_launch(L, parity, seed);
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) phase: %s", cudaGetErrorString(e));
}

int qcd_on_measure(qcd_on* L, double* out) {
  if (int rc = check(L)) return rc;
  if (!out) return fail(QCD_ERR_INVALID_ARG, "out is null");
  const OnCtx a = make_on_ctx(L, L->seed);
  if (L->precision == QCD_FP64_PLAIN)
    on_measure_kernel<double><<<L->n_meas_blocks, ON_MEAS_THREADS, 0, L->stream>>>(a);
  else
    on_measure_kernel<float><<<L->n_meas_blocks, ON_MEAS_THREADS, 0, L->stream>>>(a);
  on_measure_final<<<1, 1024, 0, L->stream>>>(a, L->n_meas_blocks);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, a.meas_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, L->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) measure: %s", cudaGetErrorString(e));
}

int qcd_on_get_field(qcd_on* L, double* host_out) {
  if (int rc = check(L)) return rc;
  if (!host_out) return fail(QCD_ERR_INVALID_ARG, "host_out is null");
  const size_t bytes = size_t(2) * L->g.Vh * L->N * sizeof(double);
  return copy_via_device(L, bytes, [&](double* d) {
    const OnCtx a = make_on_ctx(L, L->seed);
    const unsigned grid = unsigned((2LL * L->g.Vh + 255) / 256);
    if (L->precision == QCD_FP64_PLAIN) on_to_canonical<double><<<grid, 256, 0, L->stream>>>(a, d);
    else on_to_canonical<float><<<grid, 256, 0, L->stream>>>(a, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, bytes, cudaMemcpyDeviceToHost, L->stream);
    return e;
  });
}

int qcd_on_set_field(qcd_on* L, const double* host_in) {
  if (int rc = check(L)) return rc;
  if (!host_in) return fail(QCD_ERR_INVALID_ARG, "host_in is null");
  const size_t bytes = size_t(2) * L->g.Vh * L->N * sizeof(double);
  return copy_via_device(L, bytes, [&](double* d) {
    cudaError_t e = cudaMemcpyAsync(d, host_in, bytes, cudaMemcpyHostToDevice, L->stream);
    const OnCtx a = make_on_ctx(L, L->seed);
    const unsigned grid = unsigned((2LL * L->g.Vh + 255) / 256);
    if (e == cudaSuccess) {
      if (L->precision == QCD_FP64_PLAIN) on_from_canonical<double><<<grid, 256, 0, L->stream>>>(a, d);
      else on_from_canonical<float><<<grid, 256, 0, L->stream>>>(a, d);
      e = cudaGetLastError();
    }
    return e;
  });
}

int qcd_on_get_sweep(qcd_on* L, uint32_t* sweep) {
  if (int rc = check(L)) return rc;
  if (!sweep) return fail(QCD_ERR_INVALID_ARG, "sweep is null");
  cudaError_t e = cudaMemcpyAsync(sweep, L->d_small, sizeof(uint32_t), cudaMemcpyDeviceToHost, L->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) get_sweep: %s", cudaGetErrorString(e));
}

int qcd_on_set_sweep(qcd_on* L, uint32_t sweep) {
  if (int rc = check(L)) return rc;
  cudaError_t e = cudaMemcpyAsync(L->d_small, &sweep, sizeof(uint32_t), cudaMemcpyHostToDevice, L->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) set_sweep: %s", cudaGetErrorString(e));
}

int qcd_on_get_accepted(qcd_on* L, unsigned long long* accepted) {
  if (int rc = check(L)) return rc;
  if (!accepted) return fail(QCD_ERR_INVALID_ARG, "accepted is null");
  cudaError_t e =
      cudaMemcpyAsync(accepted, L->d_small + 8, sizeof(unsigned long long), cudaMemcpyDeviceToHost, L->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
  return e == cudaSuccess ? QCD_OK : fail(QCD_ERR_CUDA, "O(N) get_accepted: %s", cudaGetErrorString(e));
}

}  // extern "C"
