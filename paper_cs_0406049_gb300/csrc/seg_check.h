// seg_check.h -- the check every batched kernel applies to a descriptor
// before it touches the descriptor's arrays, also exported on the host as
// sincos_seg_check().  Plain C++ (no device code), so that host code and
// kernels share the one definition.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define SINCOS_HD __host__ __device__ __forceinline__
#else
#define SINCOS_HD inline
#endif

namespace sincos_gb300 {

// Whether one array of a batch can be processed: an array of len <= 0 needs
// nothing (its pointers are never used); otherwise x, s and c must be
// non-null, x aligned to 4 bytes and s and c to out_size (4 or 2) bytes.
// Kernels skip an array that fails and count it (sincos_device_bad_segments).
SINCOS_HD bool seg_usable(const void *x, const void *s, const void *c, int64_t len,
                          unsigned out_size)
{
    if (len <= 0) return true;
    if (!x || !s || !c) return false;
    const uintptr_t m = (uintptr_t)out_size - 1u;
    return (((uintptr_t)x & 3u) | ((uintptr_t)s & m) | ((uintptr_t)c & m)) == 0;
}

}  // namespace sincos_gb300
