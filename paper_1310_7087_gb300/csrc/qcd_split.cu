// qcd_split.cu -- link storage of a lattice divided into two parts along t:
// the first t-slices of every link array in device memory, the remaining ones
// in host memory of the CPU next to the GPU (the paper's division of a lattice
// into parts when the device memory does not hold it, Sect. "Multi-GPU Mode
// and Distributed Simulations").
//
// Both parts sit behind one contiguous virtual address range (CUDA virtual
// memory management: cuMemAddressReserve + cuMemCreate on a device location and
// on a host-NUMA location + cuMemMap), so every kernel addresses the links
// exactly as for a device-resident lattice.  On a Grace host the GPU reads and
// writes the host part coherently over NVLink-C2C: no halo copies between
// parts and no second-level checkerboard schedule are needed.
//
// The driver entry points come from cudaGetDriverEntryPointByVersion, so the
// library has no link-time dependency on libcuda.
#include "qcd.h"
#include "qcd_split.h"

#include <cuda.h>

#include <cstdio>
#include <vector>

namespace qcd {

namespace {

struct DriverVmm {
  CUresult (*getAttribute)(int*, CUdevice_attribute, CUdevice) = nullptr;
  CUresult (*granularity)(size_t*, const CUmemAllocationProp*, CUmemAllocationGranularity_flags) = nullptr;
  CUresult (*reserve)(CUdeviceptr*, size_t, size_t, CUdeviceptr, unsigned long long) = nullptr;
  CUresult (*addressFree)(CUdeviceptr, size_t) = nullptr;
  CUresult (*create)(CUmemGenericAllocationHandle*, size_t, const CUmemAllocationProp*, unsigned long long) = nullptr;
  CUresult (*release)(CUmemGenericAllocationHandle) = nullptr;
  CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long) = nullptr;
  CUresult (*unmap)(CUdeviceptr, size_t) = nullptr;
  CUresult (*setAccess)(CUdeviceptr, size_t, const CUmemAccessDesc*, size_t) = nullptr;
  bool ok = false;
};

template <typename F>
bool entry(const char* name, F& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  fn = reinterpret_cast<F>(p);
  return true;
}

const DriverVmm& vmm() {
  static const DriverVmm d = [] {
    DriverVmm v;
    v.ok = entry("cuDeviceGetAttribute", v.getAttribute) && entry("cuMemGetAllocationGranularity", v.granularity) &&
           entry("cuMemAddressReserve", v.reserve) && entry("cuMemAddressFree", v.addressFree) &&
           entry("cuMemCreate", v.create) && entry("cuMemRelease", v.release) && entry("cuMemMap", v.map) &&
           entry("cuMemUnmap", v.unmap) && entry("cuMemSetAccess", v.setAccess);
    return v;
  }();
  return d;
}

CUmemAllocationProp prop_for(bool host, int id) {
  CUmemAllocationProp p{};
  p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  p.location.type = host ? CU_MEM_LOCATION_TYPE_HOST_NUMA : CU_MEM_LOCATION_TYPE_DEVICE;
  p.location.id = id;
  return p;
}

}  // namespace

struct SplitLinks {
  CUdeviceptr va = 0;
  size_t total = 0;
  bool mapped = false;
  std::vector<CUmemGenericAllocationHandle> handles;
};

int split_host_node(int device, size_t* granularity) {
  const DriverVmm& d = vmm();
  *granularity = 0;
  if (!d.ok) return -1;
  int vmm_host = 0, numa = -1;
  if (d.getAttribute(&vmm_host, CU_DEVICE_ATTRIBUTE_HOST_NUMA_VIRTUAL_MEMORY_MANAGEMENT_SUPPORTED, device) !=
          CUDA_SUCCESS ||
      d.getAttribute(&numa, CU_DEVICE_ATTRIBUTE_HOST_NUMA_ID, device) != CUDA_SUCCESS || vmm_host != 1 || numa < 0)
    return -1;
  size_t gd = 0, gh = 0;
  const CUmemAllocationProp pd = prop_for(false, device), ph = prop_for(true, numa);
  if (d.granularity(&gd, &pd, CU_MEM_ALLOC_GRANULARITY_MINIMUM) != CUDA_SUCCESS ||
      d.granularity(&gh, &ph, CU_MEM_ALLOC_GRANULARITY_MINIMUM) != CUDA_SUCCESS || !gd || !gh)
    return -1;
  *granularity = gd > gh ? (gd % gh ? gd * gh : gd) : (gh % gd ? gd * gh : gh);
  return numa;
}

void split_free(SplitLinks* s) {
  if (!s) return;
  const DriverVmm& d = vmm();
  if (s->mapped) d.unmap(s->va, s->total);
  for (CUmemGenericAllocationHandle h : s->handles) d.release(h);
  if (s->va) d.addressFree(s->va, s->total);
  delete s;
}

// n_arrays arrays of array_bytes each, contiguous; the first device_bytes of
// every array in device memory, the rest in host memory of NUMA node `node`.
// array_bytes and device_bytes must be multiples of the granularity.  Every
// byte of the range is mapped before the range is returned.
int split_alloc(int device, int node, size_t granularity, size_t n_arrays, size_t array_bytes, size_t device_bytes,
                SplitLinks** out, void** base, char* why, size_t why_len) {
  *out = nullptr;
  *base = nullptr;
  const DriverVmm& d = vmm();
  if (!d.ok || !granularity || array_bytes % granularity || device_bytes % granularity || device_bytes > array_bytes ||
      !n_arrays) {
    snprintf(why, why_len, "split storage: bad layout (array %zu B, device part %zu B, granularity %zu B)",
             array_bytes, device_bytes, granularity);
    return QCD_ERR_INVALID_ARG;
  }
  SplitLinks* s = new SplitLinks();
  s->total = n_arrays * array_bytes;
  auto fail = [&](const char* what, CUresult r) {
    snprintf(why, why_len, "split storage: %s failed (driver error %d)", what, int(r));
    split_free(s);
    return r == CUDA_ERROR_OUT_OF_MEMORY ? QCD_ERR_OOM : QCD_ERR_CUDA;
  };
  CUresult r = d.reserve(&s->va, s->total, granularity, 0, 0);
  if (r != CUDA_SUCCESS) {
    s->va = 0;
    return fail("cuMemAddressReserve", r);
  }
  const CUmemAllocationProp pd = prop_for(false, device), ph = prop_for(true, node);
  std::vector<std::pair<size_t, size_t>> done;  // mapped (offset, size)
  for (size_t a = 0; a < n_arrays; ++a) {
    const size_t off = a * array_bytes;
    const size_t piece[2] = {device_bytes, array_bytes - device_bytes};
    size_t at = off;
    for (int k = 0; k < 2; ++k) {
      if (!piece[k]) continue;
      CUmemGenericAllocationHandle h{};
      if ((r = d.create(&h, piece[k], k ? &ph : &pd, 0)) != CUDA_SUCCESS) {
        for (auto& m : done) d.unmap(s->va + m.first, m.second);
        return fail(k ? "cuMemCreate (host part)" : "cuMemCreate (device part)", r);
      }
      s->handles.push_back(h);
      if ((r = d.map(s->va + at, piece[k], 0, h, 0)) != CUDA_SUCCESS) {
        for (auto& m : done) d.unmap(s->va + m.first, m.second);
        return fail("cuMemMap", r);
      }
      done.emplace_back(at, piece[k]);
      at += piece[k];
    }
  }
  s->mapped = true;
  CUmemAccessDesc acc{};
  acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  acc.location.id = device;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  if ((r = d.setAccess(s->va, s->total, &acc, 1)) != CUDA_SUCCESS) return fail("cuMemSetAccess", r);
  *out = s;
  *base = reinterpret_cast<void*>(s->va);
  return QCD_OK;
}

}  // namespace qcd
