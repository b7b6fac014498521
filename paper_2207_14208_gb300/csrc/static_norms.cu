// Residual norms without any device allocation.
//
// bcmg_residual_norms_static() serves callers that cannot allocate device
// memory themselves (for example code running inside a CUDA-graph capture, a
// plugin whose host application owns every allocation, or an environment that
// forbids cudaMalloc after start-up).  The caller passes the residual and
// class arrays and a 4-double device output; the per-block partial sums live
// in a fixed file-scope __device__ array instead of scratch that would have
// to be allocated.
//
// That array exists once per device that loads this library and stays
// allocated until the process exits.  Its host-side name is only a stand-in
// for the device symbol, so the first call on each device looks up the real
// device address with cudaGetSymbolAddress (with that device current) and
// caches it; make that first call before starting any stream capture.  All
// calls share the array and it keeps the last call's partial sums: calls
// that overlap on the GPU (different streams, or different host threads on
// the same device) race and must be ordered by the caller.  Nothing in the
// array has to start at zero: each call writes every slot it later reads.
#include <mutex>

#include "bcmg_internal.cuh"

namespace bcmg {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticPerThread = 32;
constexpr int64_t kStaticTile = (int64_t)kStaticThreads * kStaticPerThread;  // entries per block
constexpr int kStaticBlocks = 4096;                                            // partial-sum slots
constexpr int kMaxDevices = 64;

// 4 partials (sum r_I^2, sum r_G^2, max|r_I|, max|r_G|) per block: 128 KiB
static __device__ __align__(256) double g_norm_scratch[kStaticBlocks * 4];

std::mutex g_static_mu;
double *g_static_ptr[kMaxDevices] = {};

__global__ void __launch_bounds__(kStaticThreads) k_static_partial(const double *__restrict__ r,
                                                                   const uint8_t *__restrict__ cls, int64_t n,
                                                                   double *__restrict__ part) {
    __shared__ double sh[4][kStaticThreads];
    double sI = 0.0, sG = 0.0, mI = 0.0, mG = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kStaticTile;
    for (int i = 0; i < kStaticPerThread; ++i) {
        const int64_t x = base + (int64_t)i * kStaticThreads + threadIdx.x;
        if (x >= n) break;
        const uint8_t c = cls[x];
        const double v = r[x];
        if (c == CL_INTERIOR) {
            sI = fma(v, v, sI);
            mI = fmax(mI, fabs(v));
        } else if (c == CL_GHOST) {
            sG = fma(v, v, sG);
            mG = fmax(mG, fabs(v));
        }
    }
    sh[0][threadIdx.x] = sI;
    sh[1][threadIdx.x] = sG;
    sh[2][threadIdx.x] = mI;
    sh[3][threadIdx.x] = mG;
    __syncthreads();
    for (int s = kStaticThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[(int64_t)blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(1024) k_static_final(const double *__restrict__ part, int nparts,
                                                       double *__restrict__ out) {
    __shared__ double sh[4][1024];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a[0] += part[i * 4 + 0];
        a[1] += part[i * 4 + 1];
        a[2] = fmax(a[2], part[i * 4 + 2]);
        a[3] = fmax(a[3], part[i * 4 + 3]);
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(sh[0][0]);
        out[1] = sqrt(sh[1][0]);
        out[2] = sh[2][0];
        out[3] = sh[3][0];
    }
}

// device address of the static scratch on the current device, looked up once
int static_scratch(double **ptr, std::string *msg) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return BCMG_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *msg = "device index out of range";
        return BCMG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess || !p) {
            *msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return BCMG_ECUDA;
        }
        g_static_ptr[dev] = (double *)p;
    }
    *ptr = g_static_ptr[dev];
    return BCMG_OK;
}

}  // namespace

int static_norms(const double *r_dev, const uint8_t *cls_dev, int64_t count, double *out_dev, void *stream,
                 std::string *msg) {
    if (!r_dev || !cls_dev || !out_dev) {
        *msg = "null pointer";
        return BCMG_EINVAL;
    }
    if (count < 1 || count > kStaticTile * kStaticBlocks) {
        *msg = "count must be in [1, " + std::to_string(kStaticTile * kStaticBlocks) +
               "] (capacity of the static scratch)";
        return BCMG_EINVAL;
    }
    double *part = nullptr;
    int rc = static_scratch(&part, msg);
    if (rc != BCMG_OK) return rc;
    const int nblk = (int)((count + kStaticTile - 1) / kStaticTile);
    cudaStream_t st = (cudaStream_t)stream;
    k_static_partial<<<nblk, kStaticThreads, 0, st>>>(r_dev, cls_dev, count, part);
    k_static_final<<<1, 1024, 0, st>>>(part, nblk, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *msg = std::string("launch: ") + cudaGetErrorString(e);
        return BCMG_ECUDA;
    }
    add_launches(2);
    return BCMG_OK;
}

}  // namespace bcmg

extern "C" int bcmg_residual_norms_static(const double *r_dev, const uint8_t *cls_dev, int64_t count,
                                          double *out_dev, void *stream) {
    std::string msg;
    int rc = bcmg::static_norms(r_dev, cls_dev, count, out_dev, stream, &msg);
    return bcmg::report(rc, msg);
}
