// A caller's own kernels using the device-side point operations of
// include/gpufilter_device.cuh on filters built through the C ABI: one key
// per thread, the view passed by value.
#include <cuda_runtime.h>

#include "gpufilter_device.cuh"

__global__ void device_query_kernel(filter_device_view v, const uint64_t *keys, uint64_t n, uint8_t *found,
                                    uint64_t *counts)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (v.kind == FILTER_TCF) {
            found[i] = gf_device_tcf_contains(v, keys[i]) ? 1 : 0;
        } else {
            const uint64_t c = gf_device_gqf_count(v, keys[i]);
            if (counts) counts[i] = c;
            if (found) found[i] = c ? 1 : 0;
        }
    }
}

extern "C" int device_query_example(const filter_device_view *v, const uint64_t *keys, uint64_t n, uint8_t *found,
                                    uint64_t *counts, void *stream)
{
    if (!v || n == 0) return 0;
    const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    device_query_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(*v, keys, n, found, counts);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

__global__ void device_update_kernel(filter_device_view v, const uint64_t *keys, uint64_t n, int remove,
                                     uint8_t *status)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        int st;
        if (v.kind == FILTER_GQF) st = remove ? gf_device_gqf_remove(v, keys[i]) : gf_device_gqf_insert(v, keys[i]);
        else st = remove ? gf_device_tcf_remove(v, keys[i]) : gf_device_tcf_insert(v, keys[i]);
        if (status) status[i] = (uint8_t)st;
    }
}

extern "C" int device_update_example(const filter_device_view *v, const uint64_t *keys, uint64_t n, int remove,
                                     uint8_t *status, void *stream)
{
    if (!v || n == 0) return 0;
    const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    device_update_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(*v, keys, n, remove, status);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// TCF with values: read the smallest stored value per key, or insert keys
// with their values (point mode).
__global__ void device_value_kernel(filter_device_view v, const uint64_t *keys, uint64_t n, const uint8_t *in,
                                    uint8_t *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (in) out[i] = (uint8_t)gf_device_tcf_insert(v, keys[i], in[i]);
        else out[i] = (uint8_t)gf_device_tcf_value(v, keys[i]);
    }
}

extern "C" int device_value_example(const filter_device_view *v, const uint64_t *keys, uint64_t n,
                                    const uint8_t *values_in, uint8_t *out, void *stream)
{
    if (!v || n == 0) return 0;
    const unsigned grid = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    device_value_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(*v, keys, n, values_in, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// The same updates applied by one thread, key after key (no concurrency).
__global__ void device_update_serial_kernel(filter_device_view v, const uint64_t *keys, uint64_t n, int remove,
                                            uint8_t *status)
{
    for (uint64_t i = 0; i < n; i++) {
        int st;
        if (v.kind == FILTER_GQF) st = remove ? gf_device_gqf_remove(v, keys[i]) : gf_device_gqf_insert(v, keys[i]);
        else st = remove ? gf_device_tcf_remove(v, keys[i]) : gf_device_tcf_insert(v, keys[i]);
        if (status) status[i] = (uint8_t)st;
    }
}

extern "C" int device_update_serial_example(const filter_device_view *v, const uint64_t *keys, uint64_t n, int remove,
                                            uint8_t *status, void *stream)
{
    if (!v || n == 0) return 0;
    device_update_serial_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(*v, keys, n, remove, status);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
