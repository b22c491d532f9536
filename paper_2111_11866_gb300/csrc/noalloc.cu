// noalloc.cu -- seg4d_residual_norms_noalloc: the residual norms of a step
// system held entirely in the caller's device memory, computed without any
// device allocation.
//
// It follows the stopping test of every solve (k_defect in mixed_kernels.cu
// + k_reduce in solve_kernels.cu): per-block records followed by one
// fixed-order final reduction.  Here the per-block records live in the
// file-scope device array below instead of memory allocated by a handle, and
// the inputs are the caller's x-fastest arrays (u, b, diagonal and the 8
// off-diagonal magnitudes per voxel, as seg4d_read_field returns them).
//
// The scratch array is shared by every call in the process on a given device
// and keeps the contents of the last call.  Each call overwrites exactly the
// records it reads, so nothing has to be cleared, but calls whose work
// overlaps on the GPU (two streams, or two host threads) race on it.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/seg4d.h"
#include "seg4d_internal.cuh"

namespace {

constexpr int kRowsPerBlock = 256;                // 8 warps x 32 x-lines
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 16384;                 // records available in the scratch array
constexpr long long kMaxRows = (long long)kRowsPerBlock * kMaxBlocks;   // 4,194,304 x-lines
constexpr int kMaxDevices = 64;

// Two doubles per block: sum of r^2 and sum of b^2.  256 KiB on every device
// that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_records[2 * kMaxBlocks];

// Device address of the scratch array per device, cached once a lookup has
// succeeded; a failed lookup (for example one made during a stream capture)
// is not cached, so the next call tries again.
double *g_records_addr[kMaxDevices] = {};
std::mutex g_records_mutex[kMaxDevices];


// r_v = b_v - diag_v u_v + sum_f off[v][f] u_nb(f) over the faces whose
// neighbour lies in the grid (the Dirichlet ghost value is 0).
__global__ void __launch_bounds__(kThreads) k_residual_records(
    int n1, int n2, int n3, int n4, const float *__restrict__ u, const float *__restrict__ b,
    const float *__restrict__ diag, const float *__restrict__ off, double *__restrict__ records)
{
    const long long rows = (long long)n2 * n3 * n4;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long sy = n1, sz = (long long)n1 * n2, st = (long long)n1 * n2 * n3;
    double rr = 0.0, bb = 0.0;
    const long long row0 = (long long)blockIdx.x * kRowsPerBlock;
    for (int rw = wid; rw < kRowsPerBlock; rw += kThreads / 32) {
        const long long row = row0 + rw;
        if (row >= rows) break;
        const int j = (int)(row % n2);
        const int k = (int)((row / n2) % n3);
        const int l = (int)(row / ((long long)n2 * n3));
        for (int i = lane; i < n1; i += 32) {
            const long long v = row * n1 + i;
            const float *o = off + 8 * v;
            double acc = (double)b[v] - (double)diag[v] * (double)u[v];
            if (i > 0) acc += (double)o[0] * (double)u[v - 1];
            if (i + 1 < n1) acc += (double)o[1] * (double)u[v + 1];
            if (j > 0) acc += (double)o[2] * (double)u[v - sy];
            if (j + 1 < n2) acc += (double)o[3] * (double)u[v + sy];
            if (k > 0) acc += (double)o[4] * (double)u[v - sz];
            if (k + 1 < n3) acc += (double)o[5] * (double)u[v + sz];
            if (l > 0) acc += (double)o[6] * (double)u[v - st];
            if (l + 1 < n4) acc += (double)o[7] * (double)u[v + st];
            rr += acc * acc;
            bb += (double)b[v] * (double)b[v];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    __shared__ double sh[2][kThreads / 32];
    if (lane == 0) {
        sh[0][wid] = rr;
        sh[1][wid] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) {
            rr += sh[0][w];
            bb += sh[1][w];
        }
        records[2 * blockIdx.x] = rr;
        records[2 * blockIdx.x + 1] = bb;
    }
}

// one block: fixed-order sum of the first nblocks records
__global__ void __launch_bounds__(1024) k_records_final(const double *__restrict__ records,
                                                        int nblocks, double *__restrict__ result)
{
    double rr = 0.0, bb = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
        rr += records[2 * q];
        bb += records[2 * q + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = rr;
        sh[1][wid] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            rr += sh[0][w];
            bb += sh[1][w];
        }
        result[0] = sqrt(rr);
        result[1] = sqrt(bb);
    }
}

seg4d_status noalloc_fail(seg4d_status st, const std::string &msg)
{
    seg4d_impl::handle_free_error() = msg;
    return st;
}

}  // namespace

extern "C" seg4d_status seg4d_residual_norms_noalloc(const seg4d_dims *dims, const float *u,
                                                     const float *b, const float *diag,
                                                     const float *off, double *result,
                                                     void *cuda_stream)
{
    seg4d_impl::handle_free_error().clear();
    if (!dims || dims->n1 < 1 || dims->n2 < 1 || dims->n3 < 1 || dims->n4 < 1)
        return noalloc_fail(SEG4D_ERR_INVALID, "residual_norms_noalloc: dims must all be >= 1");
    if (!u || !b || !diag || !off || !result)
        return noalloc_fail(SEG4D_ERR_INVALID, "residual_norms_noalloc: NULL pointer");
    const long long rows = (long long)dims->n2 * dims->n3 * dims->n4;
    if (rows > kMaxRows || rows * dims->n1 >= (1LL << 33))
        return noalloc_fail(SEG4D_ERR_INVALID,
                            "residual_norms_noalloc: grid too large for its fixed scratch: "
                            "n2*n3*n4 must be <= 4194304 x-lines and n1*n2*n3*n4 < 2^33 voxels");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SEG4D_ERR_CUDA, std::string("residual_norms_noalloc: no current "
                                                        "device: ") + cudaGetErrorString(e));
    // with that device current: the device address of the scratch array (its
    // host-side name is only a stand-in), looked up until a lookup succeeds
    double *records = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_records_mutex[dev]);
        if (!g_records_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_records);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();   // the failed lookup's error is reported here, not later
                return noalloc_fail(SEG4D_ERR_CUDA,
                                    std::string("residual_norms_noalloc: scratch address: ") +
                                        cudaGetErrorString(e));
            }
            g_records_addr[dev] = (double *)p;
        }
        records = g_records_addr[dev];
    }
    const int nblocks = (int)((rows + kRowsPerBlock - 1) / kRowsPerBlock);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // an error left pending by earlier, unrelated work must not be reported
    // as this call's launch failure
    cudaGetLastError();
    k_residual_records<<<nblocks, kThreads, 0, st>>>(dims->n1, dims->n2, dims->n3, dims->n4, u, b,
                                                     diag, off, records);
    k_records_final<<<1, 1024, 0, st>>>(records, nblocks, result);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(SEG4D_ERR_CUDA, std::string("residual_norms_noalloc: launch: ") +
                                                cudaGetErrorString(e));
    return SEG4D_OK;
}
