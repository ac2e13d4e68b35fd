// qcd_batch.cu -- batched parameter scan: many independent SU(2) lattices of
// uneven sizes swept by one persistent, cooperative kernel launch that is
// captured in a CUDA graph.
//
// Each lattice owns a contiguous group of CTAs, sized in proportion to its
// work, and its phases are separated by a barrier of that group only: lattices
// never wait for one another and there is no grid-wide barrier.  A scan whose
// links outgrow L2 is swept in waves: consecutive lattices whose links fit in
// L2 (the wave budget) form one persistent launch that runs all the sweeps of
// the call, and the waves follow one another in the captured graph.  The
// lattices are independent, so each wave's links stay in L2 across its
// sweeps instead of streaming from HBM in every phase.  A group of
// one CTA synchronises with __syncthreads; larger groups use an arrival
// counter in global memory with a bounded wait (time and iteration limits):
// when it runs out the kernel records an error and returns, and the host
// reports QCD_ERR_TIMEOUT.  Links change between the phases of one launch, so
// the kernel loads them with ld.global.cg (L2 only; no stale L1 lines).
#include "qcd.h"
#include "qcd_internal.h"
#include "qcd_su2c.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace qcd {

struct BatchLat {
  int Ns, Nt, Vh, flux;
  int64_t plane;
  int64_t link_off;  // bytes from the batch's link base
  int phase_off;     // first entry of this lattice in the phase tables
  int g0, g;         // first CTA and number of CTAs of the lattice's group
  double beta;
  uint32_t kxor;     // lattice_id * 0x9E3779B9, xored into the Philox key
};

struct BatchArgs {
  const BatchLat* lat;
  const int* cta_lattice;  // CTA -> lattice
  unsigned char* links;
  const double2* phase64;
  const float2* phase32;
  unsigned* arrive;     // per-lattice arrival counters, zero at launch
  int* error;           // 1 after a wait ran out
  int* error_where;     // lattice whose wait ran out
  unsigned long long* exhausted;
  double* partials;     // 4 per CTA
  double* meas;         // [n][n_sweeps][5]
  const uint32_t* sweep0;
  uint32_t seed_lo, seed_hi;
  int nhit, n_sweeps, n_or;
  long long wait_cycles;
  int stall_lattice;    // test hook: this lattice's barriers wait for one arrival too many (-1: off)
};

constexpr int BATCH_MAX_THREADS = 512;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of one lattice's CTA group: wait until `target` arrivals.  Returns
// false if the wait ran out or another CTA already reported a failure.
__device__ bool group_barrier(const BatchArgs& b, int li, unsigned target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(b.arrive + li, 1u);
    int good = 1;
    const long long t0 = clock64();
    const long long max_iter = b.wait_cycles / 32 + 1;
    long long iter = 0;
    while (ld_acquire_u32(b.arrive + li) < target) {
      if (ld_relaxed_i32(b.error)) {
        good = 0;
        break;
      }
      if (clock64() - t0 > b.wait_cycles || ++iter > max_iter) {
        if (atomicCAS(b.error, 0, 1) == 0) *b.error_where = li;
        good = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void block_sum4(double v[4], double* out) {
  __shared__ double sh[4][BATCH_MAX_THREADS / 32];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[k][warp] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[k][w];
      out[k] = s;
    }
  }
  __syncthreads();
}

// A thread's sites h = first, first + stride, ... of one parity, walked by
// their coordinates: r = 2 h = x0 + Ns (y + Ns (z + Ns t)) (x0 even) grows by
// 2 stride per step, added digit by digit with carries, so no site costs a
// division by Ns or Nt (two thirds of the scan's lattices are not powers of
// two).  The digits of 2 first and 2 stride are found once per launch.
struct SiteWalk {
  int x0, y, z, t;  // digits of 2 h
  __device__ __forceinline__ LexSite site(int parity, int h) const {
    LexSite x;
    x.c[0] = x0 + ((parity + y + z + t) & 1);
    x.c[1] = y;
    x.c[2] = z;
    x.c[3] = t;
    x.s = 2 * h + (x.c[0] - x0);
    return x;
  }
  // d: the digits of 2 stride (d.w may exceed Nt)
  __device__ __forceinline__ void step(int Ns, const int4& d) {
    x0 += d.x;
    int c = x0 >= Ns;
    x0 -= c ? Ns : 0;
    y += d.y + c;
    c = y >= Ns;
    y -= c ? Ns : 0;
    z += d.z + c;
    c = z >= Ns;
    z -= c ? Ns : 0;
    t += d.w + c;
  }
};

// Digits (x0, y, z, t) of r = x0 + Ns (y + Ns (z + Ns t)).
__device__ inline int4 site_digits(const Geom& g, int r) {
  int4 d;
  d.x = r % g.Ns;
  r /= g.Ns;
  d.y = r % g.Ns;
  r /= g.Ns;
  d.z = r % g.Ns;
  d.w = r / g.Ns;
  return d;
}

// One phase over this CTA's share of the lattice; returns the sum of the
// updates' plaquette terms (KIND_OR_MEAS) in FP64.
// The digits of 2 stride are the same for the whole CTA: they are read from
// shared memory (d) instead of being held in registers.
template <typename R, bool FIELD, int KIND>
__device__ __forceinline__ double batch_phase(const Ctx& a, int p, int mu, int first, int stride, const int4* d,
                                              uint32_t sweep) {
  double v = 0.0;
  const int4 r0 = site_digits(a.g, 2 * first);  // once per phase: nothing held across phases
  SiteWalk w{r0.x, r0.y, r0.z, r0.w};
  switch (mu) {
#define QCD_BATCH_MU(MU)                                                                          \
  case MU:                                                                                        \
    for (int h = first; h < a.g.Vh; h += stride, w.step(a.g.Ns, *d))                                  \
      v += double(su2c_update_at<R, FIELD, KIND, MU, true>(a, p, w.site(p, h), sweep));            \
    break;
    QCD_BATCH_MU(0)
    QCD_BATCH_MU(1)
    QCD_BATCH_MU(2)
    QCD_BATCH_MU(3)
#undef QCD_BATCH_MU
  }
  return v;
}

template <typename R, bool FIELD>
__device__ void batch_run(const BatchArgs& b, int li, const BatchLat& L, int j) {
  using P = SU2Policy<R>;
  Ctx a{};
  a.links = b.links + L.link_off;
  a.g.Ns = L.Ns;
  a.g.Nt = L.Nt;
  a.g.Vh = L.Vh;
  a.g.pow2 = ((L.Ns & (L.Ns - 1)) | (L.Nt & (L.Nt - 1))) == 0
                 ? (__ffs(L.Ns) - 1) | ((__ffs(L.Nt) - 1) << 8) | (1 << 16)
                 : 0;  // the power-of-two code of geom_set_decode (no multiply-high divisions here)
  a.g.plane = L.plane;
  a.beta = L.beta;
  a.k0 = b.seed_lo ^ L.kxor;
  a.k1 = b.seed_hi;
  a.nhit = b.nhit;
  a.flux = L.flux;
  a.phase64 = b.phase64 + L.phase_off;
  a.phase32 = b.phase32 + L.phase_off;
  a.exhausted = b.exhausted;
  const int first = j * blockDim.x + threadIdx.x, stride = L.g * blockDim.x;
  __shared__ int4 step_digits;
  if (threadIdx.x == 0) step_digits = site_digits(a.g, 2 * stride);
  __syncthreads();
  const uint32_t sweep0 = *b.sweep0;
  const bool stall = li == b.stall_lattice;
  unsigned gen = 0;
  auto barrier = [&]() -> bool {
    ++gen;
    if (L.g == 1 && !stall) {
      __syncthreads();
      return true;
    }
    return group_barrier(b, li, gen * unsigned(L.g) + (stall ? 1u : 0u));
  };
  const int64_t V = 2LL * L.Vh, V3 = int64_t(L.Ns) * L.Ns * L.Ns;
  for (int s = 0; s < b.n_sweeps; ++s) {
    const uint32_t sweep = sweep0 + uint32_t(s);
    for (int p = 0; p < 2; ++p)
      for (int mu = 0; mu < 4; ++mu) {
        batch_phase<R, FIELD, KIND_HB>(a, p, mu, first, stride, &step_digits, sweep);
        if (!barrier()) return;
      }
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    // the last OR pass reunitarizes the links it updates and its odd phases
    // mu = 1..3 sum the plaquettes of the planes (mu, nu < mu), each once
    for (int o = 0; o < b.n_or; ++o)
      for (int p = 0; p < 2; ++p)
        for (int mu = 0; mu < 4; ++mu) {
          if (o < b.n_or - 1) {
            batch_phase<R, FIELD, KIND_OR>(a, p, mu, first, stride, &step_digits, sweep);
          } else if (p == 1 && mu >= 1) {
            v[mu == 3 ? 1 : 0] += batch_phase<R, FIELD, KIND_OR_MEAS>(a, p, mu, first, stride, &step_digits, sweep);
          } else {
            batch_phase<R, FIELD, KIND_OR_REUNIT>(a, p, mu, first, stride, &step_digits, sweep);
          }
          if (!barrier()) return;
        }
    if (b.n_or == 0) {  // no OR pass to carry them: reunitarization and plaquettes on their own
      for (int64_t idx = first; idx < 4 * V; idx += stride) {
        const int plane = int(idx / L.Vh), h = int(idx % L.Vh);
        su2_reunit_link<R, true>(a, plane >> 1, plane & 1, h);
      }
      if (!barrier()) return;
      for (int64_t idx = first; idx < V; idx += stride) plaquette_site<P, FIELD, true>(a, idx, v[0], v[1]);
    }
    for (int64_t idx = first; idx < V3; idx += stride) polyakov_site<P, true>(a, idx, v[2], v[3]);
    block_sum4(v, b.partials + 4 * int64_t(blockIdx.x));
    if (!barrier()) return;
    if (j == 0 && threadIdx.x == 0) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      for (int c = 0; c < L.g; ++c)
        for (int k = 0; k < 4; ++k) t[k] += __ldcg(b.partials + 4 * int64_t(L.g0 + c) + k);
      double* m = b.meas + (int64_t(li) * b.n_sweeps + s) * 5;
      m[0] = (t[0] + t[1]) / (6.0 * double(V));
      m[1] = t[0] / (3.0 * double(V));
      m[2] = t[1] / (3.0 * double(V));
      m[3] = t[2] / double(V3);
      m[4] = t[3] / double(V3);
    }
  }
}

// Register cap of the batched kernel: at 64 registers (small spills) four
// 256-thread CTAs stay resident per SM and hide the L2/HBM latency of the
// gathers (measured: 0.735 ms per sweep of the 64-lattice scan vs 0.916 ms
// uncapped).
#ifndef QCD_BATCH_MAXNREG
#define QCD_BATCH_MAXNREG 64
#endif

template <typename R>
__global__ void __maxnreg__(QCD_BATCH_MAXNREG) batch_kernel(const BatchArgs b) {
  const int li = b.cta_lattice[blockIdx.x];
  const BatchLat L = b.lat[li];
  const int j = int(blockIdx.x) - L.g0;
  if (L.flux != 0) batch_run<R, true>(b, li, L, j);
  else batch_run<R, false>(b, li, L, j);
}

__global__ void batch_advance_kernel(uint32_t* sweep, int n) { *sweep += uint32_t(n); }

__global__ void batch_phase_table_kernel(const BatchLat* lat, int n, double2* p64, float2* p32) {
  const int li = blockIdx.x;
  if (li >= n) return;
  const BatchLat L = lat[li];
  for (int x = threadIdx.x; x < L.Ns; x += blockDim.x) {
    double s, c;
    sincospi(2.0 * double(L.flux) * double(x) / (double(L.Ns) * double(L.Ns)), &s, &c);
    p64[L.phase_off + x] = make_double2(c, s);
    p32[L.phase_off + x] = make_float2(float(c), float(s));
  }
}

}  // namespace qcd

using qcd::BatchArgs;
using qcd::BatchLat;

struct BatchGraph {
  uint64_t seed;
  int n_sweeps, n_or, nhit, block, stall;
  cudaGraphExec_t exec;
};

struct qcd_batch {
  int n = 0, group = 2, precision = QCD_FP32_COMPRESSED;
  const qcd::PolicyOps* ops = nullptr;
  std::vector<BatchLat> lat;
  std::vector<int> Ns, Nt, flux;
  std::vector<double> beta;
  uint64_t seed = 0;
  int nhit = 10;
  cudaStream_t stream = nullptr;
  int device = 0;
  int block = 0;        // threads per CTA; 0 = autotune on the next sweep
  int per_sm = 0;       // resident CTAs per SM used (0 = as many as fit)
  int total_ctas = 0;   // largest grid over the waves
  size_t wave_budget = 0;            // link bytes per wave (0: one wave)
  std::vector<int> wave_l0;          // first lattice of each wave, then n
  std::vector<int> wave_cta0;        // first entry of each wave in the CTA map
  std::vector<int> wave_ctas;        // CTAs of each wave's launch
  double wait_seconds = 2.0;
  int stall_lattice = -1;
  size_t link_bytes = 0;
  int phase_entries = 0;
  unsigned char* links = nullptr;
  BatchLat* d_lat = nullptr;
  int* d_cta = nullptr;
  double2* d_phase64 = nullptr;
  float2* d_phase32 = nullptr;
  unsigned char* d_small = nullptr;  // sweep, error, error_where, exhausted
  unsigned* d_arrive = nullptr;
  double* d_partials = nullptr;
  size_t partial_ctas = 0;
  double* d_meas = nullptr;
  size_t meas_cap = 0;  // doubles
  std::vector<BatchGraph> graphs;
};

namespace {

int batch_fail(int code, const std::string& msg) { return qcd::set_last_error(code, msg.c_str()); }

#define BATCH_CUDA(call)                                                                                       \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess)                                                                                     \
      return batch_fail(QCD_ERR_CUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));            \
  } while (0)

uint32_t* d_sweep(qcd_batch* B) { return reinterpret_cast<uint32_t*>(B->d_small); }
int* d_error(qcd_batch* B) { return reinterpret_cast<int*>(B->d_small + 4); }
int* d_error_where(qcd_batch* B) { return reinterpret_cast<int*>(B->d_small + 8); }
unsigned long long* d_exhausted(qcd_batch* B) { return reinterpret_cast<unsigned long long*>(B->d_small + 16); }

void (*batch_kernel_ptr(int precision))(BatchArgs) {
  return precision == QCD_FP64_PLAIN ? qcd::batch_kernel<double> : qcd::batch_kernel<float>;
}

// Resident CTAs for a block size (cooperative launch needs all CTAs
// resident), at most `per_sm_cap` per SM when that is > 0.
int resident_ctas(qcd_batch* B, int block, int per_sm_cap) {
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_ptr(B->precision), block, 0) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm_cap > 0) per_sm = std::min(per_sm, per_sm_cap);
  return per_sm * sms;
}

// Split `capacity` CTAs over the lattices l0 .. l1-1 (one wave).  A group's
// phase lasts as long as its busiest thread, ceil(Vh / (g block)) sites, and
// the wave as long as its slowest group, so the split minimises the largest
// per-thread load: the smallest T whose groups g = ceil(Vh / (T block)) fit
// `capacity` (at least one CTA each, never more than the lattice's sites
// need).  The CTAs left over then go one at a time to the group with the
// largest load Vh / (g block).  (For the 64-lattice scan at 608 CTAs of 256
// threads a split in proportion to Vh gives 8 sites per thread at most, this
// one 7, against a mean of 5.9; the sweep time stays within 1 %: the kernel
// is held by latency and barriers more than by its busiest thread.)
// Fills g0 (relative to the wave's launch) and g, and appends the wave's
// CTA -> lattice map.  Returns the wave's CTAs.
int allocate_ctas(qcd_batch* B, int block, int capacity, int l0, int l1, std::vector<int>& cta_lattice) {
  const int n = l1 - l0;
  if (capacity < n) return 0;
  std::vector<int> cap(n), g(n);
  int64_t T = 1;
  for (int i = 0; i < n; ++i) {
    cap[i] = std::max(1, (B->lat[l0 + i].Vh + block - 1) / block);
    T = std::max<int64_t>(T, cap[i]);  // one CTA per lattice: load ceil(Vh / block)
  }
  auto groups = [&](int64_t t) {
    int64_t sum = 0;
    for (int i = 0; i < n; ++i) {
      const int64_t per = t * block;
      g[i] = int(std::min<int64_t>(cap[i], std::max<int64_t>(1, (B->lat[l0 + i].Vh + per - 1) / per)));
      sum += g[i];
    }
    return sum;
  };
  int64_t lo = 1, hi = T;  // groups(hi) = n <= capacity
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (groups(mid) <= capacity) hi = mid;
    else lo = mid + 1;
  }
  int used = int(groups(hi));
  while (used < capacity) {
    int k = -1;
    double worst = 0.0;
    for (int i = 0; i < n; ++i) {
      if (g[i] >= cap[i]) continue;
      const double load = double(B->lat[l0 + i].Vh) / double(g[i]);
      if (load > worst) {
        worst = load;
        k = i;
      }
    }
    if (k < 0) break;
    ++g[k];
    ++used;
  }
  int c0 = 0;
  for (int i = 0; i < n; ++i) {
    B->lat[l0 + i].g0 = c0;
    B->lat[l0 + i].g = g[i];
    for (int c = 0; c < g[i]; ++c) cta_lattice.push_back(l0 + i);
    c0 += g[i];
  }
  return c0;
}

// Consecutive lattices whose links fit the wave budget (at least one lattice
// per wave; budget 0: everything in one wave): the first lattice of each
// wave, then n.
std::vector<int> wave_starts(const qcd_batch* B) {
  std::vector<int> l0(1, 0);
  size_t bytes = 0;
  for (int i = 0; i < B->n; ++i) {
    const size_t b = size_t(B->ops->comps) * 8 * size_t(B->lat[i].plane) * 16;
    if (B->wave_budget && bytes > 0 && bytes + b > B->wave_budget) {
      l0.push_back(i);
      bytes = 0;
    }
    bytes += b;
  }
  l0.push_back(B->n);
  return l0;
}
void form_waves(qcd_batch* B) { B->wave_l0 = wave_starts(B); }

void drop_batch_graphs(qcd_batch* B) {
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.exec);
  B->graphs.clear();
}

// Lay out the CTA groups of every wave for `block` threads (at most `per_sm`
// CTAs per SM, 0 = as many as fit) and upload descriptors.
int configure(qcd_batch* B, int block, int per_sm = 0) {
  const int capacity = resident_ctas(B, block, per_sm);
  form_waves(B);
  std::vector<int> map;
  B->wave_cta0.clear();
  B->wave_ctas.clear();
  int largest = 0;
  for (size_t w = 0; w + 1 < B->wave_l0.size(); ++w) {
    B->wave_cta0.push_back(int(map.size()));
    const int got = allocate_ctas(B, block, capacity, B->wave_l0[w], B->wave_l0[w + 1], map);
    if (got == 0)
      return batch_fail(QCD_ERR_NOT_SUPPORTED, "wave of " + std::to_string(B->wave_l0[w + 1] - B->wave_l0[w]) +
                                                   " lattices does not fit " + std::to_string(capacity) +
                                                   " resident CTAs of " + std::to_string(block) + " threads");
    B->wave_ctas.push_back(got);
    largest = std::max(largest, got);
  }
  if (size_t(largest) > B->partial_ctas) {
    if (B->d_partials) cudaFree(B->d_partials);
    B->d_partials = nullptr;
    B->partial_ctas = 0;
    BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&B->d_partials), size_t(largest) * 4 * sizeof(double)));
    B->partial_ctas = size_t(largest);
  }
  if (B->d_cta) cudaFree(B->d_cta);
  B->d_cta = nullptr;
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&B->d_cta), map.size() * sizeof(int)));
  BATCH_CUDA(cudaMemcpyAsync(B->d_cta, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  BATCH_CUDA(cudaMemcpyAsync(B->d_lat, B->lat.data(), B->lat.size() * sizeof(BatchLat), cudaMemcpyHostToDevice,
                             B->stream));
  BATCH_CUDA(cudaStreamSynchronize(B->stream));
  B->total_ctas = largest;
  B->block = block;
  B->per_sm = per_sm;
  drop_batch_graphs(B);
  return QCD_OK;
}

BatchArgs make_args(qcd_batch* B, unsigned char* links, uint64_t seed, int n_sweeps, int n_or, double* meas,
                    unsigned long long* exhausted) {
  BatchArgs a{};
  a.lat = B->d_lat;
  a.cta_lattice = B->d_cta;
  a.links = links;
  a.phase64 = B->d_phase64;
  a.phase32 = B->d_phase32;
  a.arrive = B->d_arrive;
  a.error = d_error(B);
  a.error_where = d_error_where(B);
  a.exhausted = exhausted;
  a.partials = B->d_partials;
  a.meas = meas;
  a.sweep0 = d_sweep(B);
  a.seed_lo = uint32_t(seed);
  a.seed_hi = uint32_t(seed >> 32);
  a.nhit = B->nhit;
  a.n_sweeps = n_sweeps;
  a.n_or = n_or;
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, B->device);
  const double hz = khz > 0 ? khz * 1e3 : 2.1e9;
  a.wait_cycles = (long long)(B->wait_seconds * hz);
  a.stall_lattice = B->stall_lattice;
  return a;
}

// Enqueue one call: zero the counters, one persistent launch per wave (each
// runs all the sweeps of its lattices), the sweep counter advance.
int enqueue(qcd_batch* B, const BatchArgs& a0, cudaStream_t st, bool advance) {
  BATCH_CUDA(cudaMemsetAsync(B->d_arrive, 0, B->n * sizeof(unsigned), st));
  for (size_t w = 0; w < B->wave_ctas.size(); ++w) {
    BatchArgs a = a0;
    a.cta_lattice = B->d_cta + B->wave_cta0[w];
    void* params[] = {&a};
    BATCH_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(batch_kernel_ptr(B->precision)),
                                           dim3(B->wave_ctas[w]), dim3(B->block), params, 0, st));
  }
  if (advance) {
    qcd::batch_advance_kernel<<<1, 1, 0, st>>>(d_sweep(B), a0.n_sweeps);
    BATCH_CUDA(cudaGetLastError());
  }
  return QCD_OK;
}

int check_error(qcd_batch* B) {
  int h[2] = {0, 0};
  BATCH_CUDA(cudaMemcpyAsync(h, d_error(B), sizeof h, cudaMemcpyDeviceToHost, B->stream));
  BATCH_CUDA(cudaStreamSynchronize(B->stream));
  if (h[0]) {
    BATCH_CUDA(cudaMemsetAsync(d_error(B), 0, 2 * sizeof(int), B->stream));
    BATCH_CUDA(cudaStreamSynchronize(B->stream));
    return batch_fail(QCD_ERR_TIMEOUT, "a barrier wait of lattice " + std::to_string(h[1]) +
                                           " ran out; the sweep was abandoned part-way");
  }
  return QCD_OK;
}

// Time one sweep for each candidate launch shape (threads per CTA x resident
// CTAs per SM) on scratch copies; keep the fastest.
int batch_autotune(qcd_batch* B) {
  unsigned char* scratch = nullptr;
  double* meas = nullptr;
  unsigned long long* exh = nullptr;
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&scratch), B->link_bytes));
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&meas), size_t(B->n) * 5 * sizeof(double)));
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&exh), sizeof(unsigned long long)));
  cudaEvent_t e0, e1;
  BATCH_CUDA(cudaEventCreate(&e0));
  BATCH_CUDA(cudaEventCreate(&e1));
  int best = 0, best_per_sm = 0;
  float best_ms = 1e30f;
  const int stall = B->stall_lattice;
  B->stall_lattice = -1;
  // every shape is timed in two rounds and keeps its faster sweep, so that
  // one slow trial (a clock step, a neighbour's burst) does not pick a shape
  constexpr int kShapes = 6;
  const int shapes[kShapes][2] = {{64, 0}, {128, 0}, {256, 0}, {256, 2}, {512, 0}, {512, 1}};
  float shape_ms[kShapes];
  for (float& m : shape_ms) m = 1e30f;
  for (int round = 0; round < 2; ++round)
    for (int si = 0; si < kShapes; ++si) {
      const int block = shapes[si][0], per_sm = shapes[si][1];
      if (configure(B, block, per_sm) != QCD_OK) {
        cudaGetLastError();
        continue;
      }
      BATCH_CUDA(cudaMemcpyAsync(scratch, B->links, B->link_bytes, cudaMemcpyDeviceToDevice, B->stream));
      const BatchArgs a = make_args(B, scratch, B->seed, 1, 1, meas, exh);
      float ms = 0.f;
      bool ok = enqueue(B, a, B->stream, false) == QCD_OK;  // warm-up
      ok = ok && cudaEventRecord(e0, B->stream) == cudaSuccess;
      ok = ok && enqueue(B, a, B->stream, false) == QCD_OK;
      ok = ok && cudaEventRecord(e1, B->stream) == cudaSuccess;
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (check_error(B) != QCD_OK) ok = false;
      if (ok) shape_ms[si] = std::min(shape_ms[si], ms);
      cudaGetLastError();
    }
  for (int si = 0; si < kShapes; ++si)
    if (shape_ms[si] < best_ms) {
      best_ms = shape_ms[si];
      best = shapes[si][0];
      best_per_sm = shapes[si][1];
    }
  B->stall_lattice = stall;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(meas);
  cudaFree(exh);
  if (!best) return batch_fail(QCD_ERR_CUDA, "batch autotune: no launch shape worked");
  return configure(B, best, best_per_sm);
}

}  // namespace

extern "C" {

int qcd_batch_create(qcd_batch** out, int n, int group, const int* Ns, const int* Nt, const double* beta,
                     const int* flux, int precision, int start, uint64_t seed, void* stream) {
  if (!out) return batch_fail(QCD_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (n < 1 || !Ns || !Nt || !beta || !flux) return batch_fail(QCD_ERR_INVALID_ARG, "need n >= 1 and four arrays");
  if (group != 2) return batch_fail(QCD_ERR_NOT_SUPPORTED, "the batched sweep runs SU(2) lattices");
  if (precision != QCD_FP64_PLAIN && precision != QCD_FP32_COMPRESSED)
    return batch_fail(QCD_ERR_INVALID_ARG, "unknown precision");
  if (start != QCD_COLD && start != QCD_HOT) return batch_fail(QCD_ERR_INVALID_ARG, "unknown start");
  qcd_batch* B = new (std::nothrow) qcd_batch();
  if (!B) return batch_fail(QCD_ERR_OOM, "host allocation failed");
  auto fail = [&](int rc) {
    qcd_batch_destroy(B);
    return rc;
  };
  B->n = n;
  B->group = group;
  B->precision = precision;
  B->ops = precision == QCD_FP64_PLAIN ? &qcd::kOpsSU2F64 : &qcd::kOpsSU2F32;
  B->seed = seed;
  B->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&B->device) != cudaSuccess) return fail(batch_fail(QCD_ERR_CUDA, "cudaGetDevice failed"));
  int l2 = 0;  // default wave budget: the device's L2
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, B->device) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  B->wave_budget = size_t(std::max(l2, 0));
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    if (Ns[i] < 2 || Nt[i] < 2 || (Ns[i] & 1) || (Nt[i] & 1))
      return fail(batch_fail(QCD_ERR_INVALID_ARG, "lattice " + std::to_string(i) + ": Ns, Nt must be even, >= 2"));
    if (!(beta[i] >= 0.0)) return fail(batch_fail(QCD_ERR_INVALID_ARG, "beta must be >= 0"));
    const long long V = (long long)Ns[i] * Ns[i] * Ns[i] * Nt[i];
    // the batched kernel indexes a lattice's FP32 link arrays (8 arrays of
    // V/2 + padding float4 each) in 32-bit arithmetic: fewer than 2^29 sites
    if (V >= (precision == QCD_FP32_COMPRESSED ? (1LL << 29) : (1LL << 31)))
      return fail(batch_fail(QCD_ERR_INVALID_ARG,
                             "lattice " + std::to_string(i) + " too large for a batch (2^29 sites FP32, 2^31 FP64)"));
    BatchLat L{};
    L.Ns = Ns[i];
    L.Nt = Nt[i];
    L.Vh = int(V / 2);
    L.flux = flux[i];
    L.plane = (L.Vh + 63) / 64 * 64;
    L.link_off = off;
    L.phase_off = B->phase_entries;
    L.beta = beta[i];
    L.kxor = uint32_t(i) * 0x9E3779B9u;
    off += int64_t(B->ops->comps) * 8 * L.plane * 16;
    B->phase_entries += Ns[i];
    B->lat.push_back(L);
    B->Ns.push_back(Ns[i]);
    B->Nt.push_back(Nt[i]);
    B->flux.push_back(flux[i]);
    B->beta.push_back(beta[i]);
  }
  B->link_bytes = size_t(off);
  if (cudaMalloc(reinterpret_cast<void**>(&B->links), B->link_bytes) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&B->d_lat), n * sizeof(BatchLat)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&B->d_phase64), B->phase_entries * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&B->d_phase32), B->phase_entries * sizeof(float2)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&B->d_small), 64) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&B->d_arrive), n * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return fail(batch_fail(QCD_ERR_OOM, "device allocation of " + std::to_string(B->link_bytes) + " bytes failed"));
  }
  cudaError_t e = cudaMemsetAsync(B->d_small, 0, 64, B->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_lat, B->lat.data(), n * sizeof(BatchLat), cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) {
    qcd::batch_phase_table_kernel<<<n, 64, 0, B->stream>>>(B->d_lat, n, B->d_phase64, B->d_phase32);
    e = cudaGetLastError();
  }
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    qcd::Ctx a{};
    a.links = B->links + B->lat[i].link_off;
    a.g = {B->lat[i].Ns, B->lat[i].Nt, B->lat[i].Vh, 0, B->lat[i].plane};
    a.k0 = uint32_t(seed) ^ B->lat[i].kxor;
    a.k1 = uint32_t(seed >> 32);
    e = B->ops->start(a, start, B->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return fail(batch_fail(QCD_ERR_CUDA, std::string("batch create: ") + cudaGetErrorString(e)));
  *out = B;
  return QCD_OK;
}

int qcd_batch_destroy(qcd_batch* B) {
  if (!B) return QCD_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  else cudaDeviceSynchronize();
  drop_batch_graphs(B);
  cudaFree(B->links);
  cudaFree(B->d_lat);
  cudaFree(B->d_cta);
  cudaFree(B->d_phase64);
  cudaFree(B->d_phase32);
  cudaFree(B->d_small);
  cudaFree(B->d_arrive);
  cudaFree(B->d_partials);
  cudaFree(B->d_meas);
  delete B;
  return QCD_OK;
}

int qcd_batch_set_block(qcd_batch* B, int threads) {
  if (!B) return batch_fail(QCD_ERR_INVALID_ARG, "null batch");
  if (threads == 0) {
    B->block = 0;
    return QCD_OK;
  }
  if (threads != 64 && threads != 128 && threads != 256 && threads != 512)
    return batch_fail(QCD_ERR_INVALID_ARG, "threads must be 0 (autotune), 64, 128, 256 or 512");
  return configure(B, threads);
}

int qcd_batch_set_wave_bytes(qcd_batch* B, size_t bytes) {
  if (!B) return batch_fail(QCD_ERR_INVALID_ARG, "null batch");
  B->wave_budget = bytes;
  if (B->block == 0) return QCD_OK;  // laid out with the launch shape on the next sweep
  return configure(B, B->block, B->per_sm);
}

int qcd_batch_get_waves(qcd_batch* B, int* waves, size_t* bytes) {
  if (!B || !waves || !bytes) return batch_fail(QCD_ERR_INVALID_ARG, "null argument");
  *waves = int(wave_starts(B).size()) - 1;
  *bytes = B->wave_budget;
  return QCD_OK;
}

int qcd_batch_get_shape(qcd_batch* B, int* threads, int* ctas) {
  if (!B || !threads || !ctas) return batch_fail(QCD_ERR_INVALID_ARG, "null argument");
  *threads = B->block;
  *ctas = B->total_ctas;
  return QCD_OK;
}

int qcd_batch_set_wait(qcd_batch* B, double seconds) {
  if (!B || !(seconds > 0.0) || seconds > 60.0) return batch_fail(QCD_ERR_INVALID_ARG, "wait must be in (0, 60] s");
  B->wait_seconds = seconds;
  drop_batch_graphs(B);
  return QCD_OK;
}

int qcd_batch_inject_stall(qcd_batch* B, int lattice) {
  if (!B || lattice < -1 || lattice >= B->n) return batch_fail(QCD_ERR_INVALID_ARG, "lattice out of range");
  B->stall_lattice = lattice;
  drop_batch_graphs(B);
  return QCD_OK;
}

int qcd_batch_sweep(qcd_batch* B, int n_sweeps, int n_overrelax, uint64_t seed, double* meas_out) {
  if (!B) return batch_fail(QCD_ERR_INVALID_ARG, "null batch");
  if (n_sweeps < 0 || n_overrelax < 0) return batch_fail(QCD_ERR_INVALID_ARG, "negative count");
  if (n_sweeps == 0) return QCD_OK;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || (cur != B->device && cudaSetDevice(B->device) != cudaSuccess))
    return batch_fail(QCD_ERR_CUDA, "cannot select the batch's device");
  if (B->block == 0)
    if (int rc = batch_autotune(B)) return rc;
  const size_t need = size_t(B->n) * size_t(n_sweeps) * 5;
  if (need > B->meas_cap) {
    if (B->d_meas) cudaFree(B->d_meas);
    B->d_meas = nullptr;
    B->meas_cap = 0;
    drop_batch_graphs(B);
    BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&B->d_meas), need * sizeof(double)));
    B->meas_cap = need;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : B->graphs)
    if (g.seed == seed && g.n_sweeps == n_sweeps && g.n_or == n_overrelax && g.nhit == B->nhit &&
        g.block == B->block && g.stall == B->stall_lattice)
      exec = g.exec;
  if (!exec) {
    if (B->graphs.size() >= 8) drop_batch_graphs(B);
    const BatchArgs a = make_args(B, B->links, seed, n_sweeps, n_overrelax, B->d_meas, d_exhausted(B));
    cudaStream_t cap;
    BATCH_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = QCD_OK;
    if (e == cudaSuccess) {
      rc = enqueue(B, a, cap, true);
      e = cudaStreamEndCapture(cap, &graph);
    }
    cudaStreamDestroy(cap);
    if (rc != QCD_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != QCD_OK ? rc : batch_fail(QCD_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return batch_fail(QCD_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    B->graphs.push_back({seed, n_sweeps, n_overrelax, B->nhit, B->block, B->stall_lattice, exec});
  }
  BATCH_CUDA(cudaGraphLaunch(exec, B->stream));
  if (int rc = check_error(B)) return rc;
  if (meas_out)
    BATCH_CUDA(cudaMemcpyAsync(meas_out, B->d_meas, need * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
  BATCH_CUDA(cudaStreamSynchronize(B->stream));
  return QCD_OK;
}

int qcd_batch_get_links(qcd_batch* B, int index, double* host_out) {
  if (!B || !host_out || index < 0 || index >= B->n) return batch_fail(QCD_ERR_INVALID_ARG, "bad argument");
  const BatchLat& L = B->lat[index];
  const size_t bytes = size_t(2) * L.Vh * 4 * 4 * 2 * sizeof(double);
  double* tmp = nullptr;
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&tmp), bytes));
  qcd::Ctx a{};
  a.links = B->links + L.link_off;
  a.g = {L.Ns, L.Nt, L.Vh, 0, L.plane};
  cudaError_t e = B->ops->to_canonical(a, tmp, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, bytes, cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return batch_fail(QCD_ERR_CUDA, std::string("batch get_links: ") + cudaGetErrorString(e));
  return QCD_OK;
}

int qcd_batch_set_links(qcd_batch* B, int index, const double* host_in) {
  if (!B || !host_in || index < 0 || index >= B->n) return batch_fail(QCD_ERR_INVALID_ARG, "bad argument");
  const BatchLat& L = B->lat[index];
  const size_t bytes = size_t(2) * L.Vh * 4 * 4 * 2 * sizeof(double);
  double* tmp = nullptr;
  BATCH_CUDA(cudaMalloc(reinterpret_cast<void**>(&tmp), bytes));
  qcd::Ctx a{};
  a.links = B->links + L.link_off;
  a.g = {L.Ns, L.Nt, L.Vh, 0, L.plane};
  cudaError_t e = cudaMemcpyAsync(tmp, host_in, bytes, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = B->ops->from_canonical(a, tmp, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return batch_fail(QCD_ERR_CUDA, std::string("batch set_links: ") + cudaGetErrorString(e));
  return QCD_OK;
}

int qcd_batch_get_sweep(qcd_batch* B, uint32_t* sweep) {
  if (!B || !sweep) return batch_fail(QCD_ERR_INVALID_ARG, "bad argument");
  BATCH_CUDA(cudaMemcpyAsync(sweep, d_sweep(B), sizeof(uint32_t), cudaMemcpyDeviceToHost, B->stream));
  BATCH_CUDA(cudaStreamSynchronize(B->stream));
  return QCD_OK;
}

int qcd_batch_link_bytes(const qcd_batch* B, size_t* bytes) {
  if (!B || !bytes) return batch_fail(QCD_ERR_INVALID_ARG, "bad argument");
  *bytes = B->link_bytes;
  return QCD_OK;
}

}  // extern "C"
