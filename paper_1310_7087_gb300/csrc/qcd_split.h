// qcd_split.h -- link storage divided along t into a device part and a host
// part behind one virtual address range (qcd_split.cu).
#pragma once

#include <cstddef>

namespace qcd {

// The host NUMA node next to `device` and the mapping granularity, or -1 when
// the device cannot map host memory this way.
struct SplitLinks;
int split_host_node(int device, size_t* granularity);
// Returns a QCD_* code and, on failure, a message in why.
int split_alloc(int device, int node, size_t granularity, size_t n_arrays, size_t array_bytes, size_t device_bytes,
                SplitLinks** out, void** base, char* why, size_t why_len);
void split_free(SplitLinks* s);

}  // namespace qcd
