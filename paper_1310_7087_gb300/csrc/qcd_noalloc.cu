// qcd_noalloc.cu -- plaquette / Polyakov-loop measurement that allocates
// nothing.
//
// Some callers cannot let this library call cudaMalloc: a host framework that
// owns all device memory through its own pool (an extra driver allocation
// either fails under the pool's memory cap or synchronizes the device in the
// middle of the framework's stream work), or code that must not have an
// allocation-failure path at all.  For them the measurement runs on a link
// buffer the caller already has, and keeps its reduction scratch in one
// file-scope device array instead of memory allocated per lattice.
#include "qcd.h"
#include "qcd_internal.h"

#include <cstring>
#include <mutex>
#include <string>

namespace {

// Block partials, the five results and the background-phase tables of the
// allocation-free measurement.  Every GPU that loads the library holds one
// copy until the process exits; all calls on that GPU share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QCD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

int noalloc_error(int code, const std::string& msg) { return qcd::set_last_error(code, msg.c_str()); }

// Layout inside the scratch array (byte offsets).
constexpr size_t kMeasOff = 0;      // 5 doubles
constexpr size_t kPhaseOff = 64;    // 4 Ns double2, then 4 Ns float2
size_t partials_offset(int Ns) { return (kPhaseOff + size_t(Ns) * 96 + 255) / 256 * 256; }

// The background tables a lattice keeps (Ctx::phase64 / phase32): the
// lambda3 phase per x, then the SU(3) diagonal of B_y with its lambda8 part,
// theta = 2 pi x / Ns^2 (n + n8, -n + n8, -2 n8).
__global__ void noalloc_phase_table(double2* p64, float2* p32, int Ns, int flux, int flux8) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Ns) return;
  const double unit = 2.0 * double(x) / (double(Ns) * double(Ns));
  double s, c;
  sincospi(double(flux) * unit, &s, &c);
  p64[x] = make_double2(c, s);
  p32[x] = make_float2(float(c), float(s));
  const int h[3] = {flux + flux8, -flux + flux8, -2 * flux8};
  for (int k = 0; k < 3; ++k) {
    sincospi(double(h[k]) * unit, &s, &c);
    p64[Ns + 3 * x + k] = make_double2(c, s);
    p32[Ns + 3 * x + k] = make_float2(float(c), float(s));
  }
}

// Device address of the scratch array on the current device; looked up once
// per device (with that device current) and cached.  The address belongs to
// the device's CUDA context: a cudaDeviceReset ends that context (and every
// lattice of this library on it), so no call may follow one in the same
// process.
int scratch_on_device(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices)
    return noalloc_error(QCD_ERR_NOT_SUPPORTED, "device index out of range for the allocation-free measurement");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_dev[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_error(QCD_ERR_CUDA, std::string("cudaGetSymbolAddress of the measurement scratch failed: ") +
                                             cudaGetErrorString(e));
    g_noalloc_dev[device] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_dev[device]);
  return QCD_OK;
}

}  // namespace

extern "C" int qcd_measure_noalloc(const void* links, size_t link_bytes, int group, int precision, int Ns, int Nt,
                                   int flux, int flux8, double* plaquette, double* polyakov, void* stream) {
  if (!links) return noalloc_error(QCD_ERR_INVALID_ARG, "links is null");
  if (group != 2 && group != 3) return noalloc_error(QCD_ERR_INVALID_ARG, "group must be 2 or 3");
  if (group == 2 && flux8 != 0) return noalloc_error(QCD_ERR_INVALID_ARG, "the lambda8 flux needs SU(3)");
  if (precision != QCD_FP64_PLAIN && precision != QCD_FP32_COMPRESSED)
    return noalloc_error(QCD_ERR_INVALID_ARG, "unknown precision");
  if (Ns < 2 || Nt < 2 || (Ns & 1) || (Nt & 1))
    return noalloc_error(QCD_ERR_INVALID_ARG, "Ns and Nt must be even and >= 2");
  const long long V = (long long)Ns * Ns * Ns * Nt;
  if (V >= (1LL << 31) || Ns > 1290) return noalloc_error(QCD_ERR_INVALID_ARG, "lattice too large");

  const qcd::PolicyOps* ops = group == 2 ? (precision == QCD_FP64_PLAIN ? &qcd::kOpsSU2F64 : &qcd::kOpsSU2F32)
                                         : (precision == QCD_FP64_PLAIN ? &qcd::kOpsSU3F64 : &qcd::kOpsSU3F32);
  qcd::GeomH g{};
  g.Ns = Ns;
  g.Nt = Nt;
  g.Vh = int(V / 2);
  qcd::geom_set_decode(g);
  // The storage holds comps x 4 directions x 2 parities arrays of `plane`
  // 16-byte vectors each; the padding of `plane` depends on how the lattice
  // was made, so it is read off the buffer size.
  const size_t arrays = size_t(ops->comps) * 8;
  if (link_bytes % (arrays * 16) != 0 || link_bytes / (arrays * 16) < size_t(g.Vh))
    return noalloc_error(QCD_ERR_INVALID_ARG,
                         std::to_string(link_bytes) + " bytes is not link storage of an SU(" +
                             std::to_string(group) + ") " + std::to_string(Ns) + "^3x" + std::to_string(Nt) +
                             " lattice (" + std::to_string(arrays) + " arrays of at least " + std::to_string(g.Vh) +
                             " 16-byte vectors each)");
  g.plane = int64_t(link_bytes / (arrays * 16));
  const size_t need = partials_offset(Ns) + qcd::measure_partials(g) * sizeof(double);
  if (need > QCD_NOALLOC_SCRATCH_BYTES)
    return noalloc_error(QCD_ERR_INVALID_ARG,
                         "lattice " + std::to_string(Ns) + "^3x" + std::to_string(Nt) + " needs " +
                             std::to_string(need) + " bytes of measurement scratch; the allocation-free "
                             "measurement has " + std::to_string(QCD_NOALLOC_SCRATCH_BYTES) +
                             " (every lattice of at most 4194304 sites, such as 64^3x16, fits)");

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return noalloc_error(QCD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  if (int rc = scratch_on_device(device, &base)) return rc;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  qcd::Ctx a{};
  a.links = const_cast<void*>(links);  // the measurement kernels only read the links
  a.g = g;
  a.flux = flux;
  a.flux8 = flux8;
  a.phase64 = reinterpret_cast<double2*>(base + kPhaseOff);
  a.phase32 = reinterpret_cast<float2*>(base + kPhaseOff + size_t(Ns) * 64);
  a.partials = reinterpret_cast<double*>(base + partials_offset(Ns));
  a.meas_out = reinterpret_cast<double*>(base + kMeasOff);

  // Nothing in the array has to start at zero: the phase table, every block
  // partial and the five results are written before they are read.
  noalloc_phase_table<<<(Ns + 63) / 64, 64, 0, st>>>(const_cast<double2*>(a.phase64),
                                                      const_cast<float2*>(a.phase32), Ns, flux, flux8);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return noalloc_error(QCD_ERR_CUDA, std::string("phase table: ") + cudaGetErrorString(e));
  if ((e = ops->measure(a, 1, st)) != cudaSuccess)
    return noalloc_error(QCD_ERR_CUDA, std::string("measure: ") + cudaGetErrorString(e));
  double h[5];
  if ((e = cudaMemcpyAsync(h, a.meas_out, sizeof h, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return noalloc_error(QCD_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  if (plaquette) std::memcpy(plaquette, h, 3 * sizeof(double));
  if (polyakov) std::memcpy(polyakov, h + 3, 2 * sizeof(double));
  return QCD_OK;
}
