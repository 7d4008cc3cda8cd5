// rsgm_window_offsets_noalloc: the ragged-volume offset computation (the
// exclusive prefix sum of the per-pixel window widths) for callers that must
// not allocate device memory.  Its scratch (row totals and row bases) is a
// file-scope device array of fixed size instead of a cudaMalloc'd buffer.
#include <mutex>

#include "rsgm_internal.cuh"


namespace {

constexpr int kMaxRows = 65536;

// Row totals [0, kMaxRows) and row bases [kMaxRows, 2 kMaxRows).  Every GPU
// that loads the library holds these 512 KiB until the process exits.  In
// host code the name below is only a stand-in; the device address comes from
// cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) uint32_t g_offset_scratch[2 * kMaxRows];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_offset_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (uint32_t *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Exclusive scan of one value per thread over a 256-thread block; the block
// total goes to `total` (shared).
__device__ __forceinline__ unsigned scan256(unsigned v, unsigned &total)
{
    __shared__ unsigned warp_pre[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) warp_pre[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const unsigned w = lane < 8 ? warp_pre[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        const unsigned tot = __shfl_sync(0xffffffffu, wi, 7);
        if (lane < 8) warp_pre[lane] = wi - w;
        if (lane == 0) total = tot;
    }
    __syncthreads();
    const unsigned res = warp_pre[wid] + incl - v;
    __syncthreads();
    return res;
}

// One block per row: in-row exclusive prefix of the widths into `offsets`,
// the row total into the scratch.
__global__ void __launch_bounds__(256) k_row_prefix(const uint32_t *__restrict__ win, int width,
                                                    uint32_t *__restrict__ offsets,
                                                    uint32_t *__restrict__ row_total)
{
    __shared__ unsigned total;
    const long long base = (long long)blockIdx.x * width;
    const int chunk = (width + blockDim.x - 1) / blockDim.x;
    const int x0 = threadIdx.x * chunk, x1 = min(width, x0 + chunk);
    unsigned local = 0;
    for (int x = x0; x < x1; ++x) local += win[base + x] >> 16;
    unsigned pre = scan256(local, total);
    for (int x = x0; x < x1; ++x) {
        offsets[base + x] = pre;
        pre += win[base + x] >> 16;
    }
    if (threadIdx.x == 0) row_total[blockIdx.x] = total;
}

// One block: exclusive scan of the row totals into the row bases.
__global__ void __launch_bounds__(256) k_row_bases(const uint32_t *__restrict__ row_total,
                                                   uint32_t *__restrict__ row_base, int rows,
                                                   uint32_t *__restrict__ total_out)
{
    __shared__ unsigned total;
    const int chunk = (rows + blockDim.x - 1) / blockDim.x;
    const int r0 = threadIdx.x * chunk, r1 = min(rows, r0 + chunk);
    unsigned local = 0;
    for (int r = r0; r < r1; ++r) local += row_total[r];
    unsigned pre = scan256(local, total);
    for (int r = r0; r < r1; ++r) {
        row_base[r] = pre;
        pre += row_total[r];
    }
    if (threadIdx.x == 0 && total_out) *total_out = total;
}

__global__ void __launch_bounds__(256) k_add_base(uint32_t *__restrict__ offsets,
                                                  const uint32_t *__restrict__ row_base, int width,
                                                  long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) offsets[i] += row_base[i / width];
}

}  // namespace

extern "C" int rsgm_window_offsets_noalloc(const uint32_t *windows, int32_t width, int32_t rows,
                                           uint32_t *offsets, uint32_t *total, void *cuda_stream)
{
    using rsgm::record_error;
    if (!windows || !offsets) return record_error(RSGM_ERR_INVALID_ARG, "NULL windows or offsets");
    if (width < 1 || width > 65535)
        return record_error(RSGM_ERR_INVALID_ARG, "width must be in [1, 65535]");
    if (rows < 1 || rows > kMaxRows)
        return record_error(RSGM_ERR_INVALID_ARG, "rows must be in [1, 65536]: the fixed scratch holds 65536 rows");
    uint32_t *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return record_error(RSGM_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t *row_total = scratch, *row_base = scratch + kMaxRows;
    const long long n = (long long)width * rows;
    k_row_prefix<<<(unsigned)rows, 256, 0, st>>>(windows, width, offsets, row_total);
    k_row_bases<<<1, 256, 0, st>>>(row_total, row_base, rows, total);
    k_add_base<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(offsets, row_base, width, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(RSGM_ERR_CUDA, cudaGetErrorString(e));
    return RSGM_OK;
}
