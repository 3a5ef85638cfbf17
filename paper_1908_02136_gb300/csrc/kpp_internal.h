// kpp_internal.h -- declarations shared by the host-side translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kpp_device.cuh"

namespace kpp {

// One streamed-form specialisation chosen for (dtype, d, lanes).
struct StreamedKernel {
    const void *fn;
    int rows_align; // per-CTA row ranges are multiples of this
    int lanes;      // lanes per row (0 for the generic kernel)
    bool generic;
};

bool streamed_lookup(int dt, int d, int lanes, StreamedKernel *out);
int streamed_threads();
int streamed_segments();
size_t streamed_smem(const StreamedKernel &k, int d);
cudaError_t streamed_launch(const StreamedKernel &k, int grid, const Problem &p, int m,
                            cudaStream_t stream);
// Point-sharded seeding (kpp_shard_*): first seed, draw after a pass, phi.
cudaError_t shard_first_launch(const Problem &p, int64_t row0, long long *xchg, int eb,
                               cudaStream_t stream);
cudaError_t shard_pick_launch(const Problem &p, int m, int rank, int world, const float *totals,
                              int64_t row0, long long *xchg, int eb, cudaStream_t stream);
cudaError_t shard_phi_launch(const float *totals, int world, double *phi, cudaStream_t stream);

// Small form (kpp_small.cu): one CTA, everything in shared memory.
const void *small_lookup(int dt, int d);
int small_threads();
size_t small_smem(int64_t N, int d, int dt);
cudaError_t small_launch(const void *fn, size_t smem, const Problem &p, cudaStream_t stream);

// Runtime arguments of the persistent kernel.
struct PersistArgs {
    int64_t cache_supers; // super-iterations of each warp's segment kept in smem
    int32_t reverse;     // walk rows backwards on odd passes
    int32_t l2_hint;     // global point loads: 0 none, 1 evict_last, 2 evict_first
    uint64_t timeout_ns; // bound of every grid-barrier wait
};

struct PersistentKernel {
    const void *fn_smem;   // D^2 in shared memory
    const void *fn_global; // D^2 in the output array
    int rows_align;          // rows per super-iteration; blocks are multiples of it
    int row_bytes;
    int lanes;
};

bool persistent_lookup(int dt, int d, int lanes, PersistentKernel *out);
int persistent_threads();
int persistent_max_blocks();
int persistent_segments();
cudaError_t persistent_launch(const void *fn, int grid, size_t smem, const Problem &p,
                              const PersistArgs &a, cudaStream_t stream);

// The options the autotuner (kpp_tune) recorded for this shape on the
// current device, if `asked` leaves every knob to the automatic choice.
bool tuned_options(int64_t N, int32_t d, int32_t K, int dt, const kpp_options &asked,
                   kpp_options *out);

} // namespace kpp

namespace kpp {

// kpp_lloyd_assign for centres whose first row and count are known only on
// the device: rows [*row0, *row0 + *kdev) of `centres` (*kdev <= kmax; 0 is
// a no-op), for points prepared by kpp_lloyd_prepare(..., kmax, ...).
kpp_status lloyd_assign_device_count(const float *centres, const long long *row0,
                                     const int32_t *kdev, int32_t kmax, int64_t N, int32_t d,
                                     int32_t *labels_out, void *workspace, size_t workspace_bytes,
                                     cudaStream_t stream);

cudaError_t quantize_bf16(const float *x, int64_t n, uint16_t *out, cudaStream_t stream);
cudaError_t quantize_fp8(const float *x, int64_t N, int d, uint8_t *q, float *scales,
                         cudaStream_t stream);

} // namespace kpp
