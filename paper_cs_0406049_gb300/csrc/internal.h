// internal.h -- host-side declarations shared by the library's translation
// units.  Not part of the public ABI (that is include/sincos_pairs.h).
#pragma once

#include <initializer_list>

#include <cuda_runtime.h>
#include <stdint.h>

#include "sincos_pairs.h"

namespace sincos_gb300 {

// Cached facts about one CUDA device.
struct DeviceInfo {
    int ordinal = -1;
    int sms = 0;
    int major = 0, minor = 0;
    int max_threads_per_sm = 0;
    // The device reads and writes pageable host memory coherently, through
    // the host's page tables (cudaDevAttrPageableMemoryAccess; Grace systems
    // over NVLink-C2C).
    bool pageable_access = false;
    char name[256] = {0};
};

// The calling thread's current device (cached per ordinal).  Returns
// SINCOS_OK and sets *info, or an error status (unsupported GPU, CUDA error).
int current_device(const DeviceInfo **info);

// Record a failed CUDA call for sincos_last_error(); returns SINCOS_ECUDA.
int cuda_fail(cudaError_t e, const char *what);
// Record `what` for sincos_last_error() and return `status` (errors that are
// not CUDA failures but need more words than the status code).
int fail_with(int status, const char *what);
// cudaGetLastError() after a launch, mapped to a status.
int check_launch(const char *what);
// Count `k` kernel launches (sincos_launch_count()).
void count_launches(uint64_t k);

// Resident CTAs per SM of `kernel` at `block` threads (cached), capped by the
// plan's request; at least 1 when the kernel fits at all, 0 when it does not.
int resident_ctas(const void *kernel, int block, int want);
// The plan with its CTA size halved (down to 32 threads) until `kernel` fits
// on an SM at all; *per_sm receives the resident CTAs per SM to size the grid
// for (0 if nothing fits).
sincos_plan fit_plan(const void *kernel, const sincos_plan &plan, int *per_sm);

bool valid_dtype(int d);
bool valid_reduction(int r);
bool valid_coef(int c);
inline int dtype_size(int d) { return d == SINCOS_F32 ? 4 : 2; }

// Plan lookup (tuned or default) for the current device.
sincos_plan plan_for(const DeviceInfo &dev, int op, int dtype, int64_t n);
bool plan_valid(const sincos_plan &p);
// The plan's forward path: 0 = bulk (TMA-staged) kernel, 16 or 32 = register
// path with that many bytes per thread per output vector.
// Whether p is a multiple of `bytes` (a power of two): element alignment of
// the arrays the entry points take (floats 4, 16-bit outputs 2).
inline bool aligned_to(const void *p, size_t bytes)
{
    return ((uintptr_t)p & (bytes - 1)) == 0;
}

// Every non-null pointer of the list aligned to 4 bytes.
inline bool all_float_aligned(std::initializer_list<const void *> ps)
{
    for (const void *p : ps)
        if (p && !aligned_to(p, 4)) return false;
    return true;
}

// Whether byte ranges [a, a + abytes) and [b, b + bbytes) share a byte.
inline bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes)
{
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + abytes;
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + bbytes;
    return a0 < b1 && b0 < a1;
}

inline int plan_vec_bytes(const sincos_plan &p) { return p.vec_bytes == 0 ? 0 : p.vec_bytes == 16 ? 16 : 32; }
// The register-path width for kernels without a bulk variant.
inline int reg_vec_bytes(const sincos_plan &p) { return p.vec_bytes == 32 ? 32 : 16; }
// Opt a kernel into `smem` bytes of dynamic shared memory (once per kernel and
// device) and return its resident CTAs per SM at that size.
int bulk_resident_ctas(const void *kernel, int block, size_t smem);
// Bounded waits that gave up in bulk kernels, per translation unit (each
// read clears the count).
unsigned take_timeouts_forward_f32();
unsigned take_timeouts_forward_bf16();
unsigned take_timeouts_forward_f16();
unsigned take_timeouts_batched_f32();
unsigned take_timeouts_batched_bf16();
unsigned take_timeouts_batched_f16();
unsigned take_timeouts_expi();
// Batched arrays skipped for a descriptor that failed seg_usable, per
// translation unit (each read clears the count).
unsigned take_bad_segments_batched_f32();
unsigned take_bad_segments_batched_bf16();
unsigned take_bad_segments_batched_f16();

// Kernel launchers.  Arguments are already validated; they enqueue on `st`
// and return a status.
int launch_forward(const float *x, void *s, void *c, int64_t n, int dtype, int red, int coef,
                   bool in_place, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st);
int launch_expi(const float *x, float *z, int64_t n, int red, int coef, const sincos_plan &plan,
                const DeviceInfo &dev, cudaStream_t st);
int launch_huygens(const float *px, const float *py, const float *pz, int64_t m,
                   const float *qx, const float *qy, const float *qz, const float *ar,
                   const float *ai, int64_t n, float k, int red, float *u,
                   const sincos_plan &plan, cudaStream_t st);
int launch_backward(const float *gs, const float *gc, const float *s, const float *c, float *gx,
                    int64_t n, bool in_place, const sincos_plan &plan, const DeviceInfo &dev,
                    cudaStream_t st);
// Batched schedule scratch, int64 of device memory: prefix[0 .. count] (tiles
// before each segment), then first_tile[0 .. G] and first_seg[0 .. G] for the
// G <= kMaxBatchedCtas CTAs of the tile kernel.
constexpr int kMaxBatchedCtas = 4096;
inline size_t batched_scratch_elems(int count)
{
    return (size_t)count + 1 + 2 * ((size_t)kMaxBatchedCtas + 1);
}

// Batched: schedule kernel over lens into `sched` (batched_scratch_elems(count)
// int64 of device scratch), then the persistent tile kernel.
int launch_batched(const sincos_seg *segs, const int64_t *lens, int count, int dtype, int red,
                   int coef, int64_t *sched, const sincos_plan &plan, const DeviceInfo &dev,
                   cudaStream_t st);


}  // namespace sincos_gb300
