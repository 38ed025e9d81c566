// ftcj_potential_noalloc: the potential and energy step for callers that
// cannot allocate device memory.  It needs no plan and calls no cudaMalloc,
// cudaFree or allocating library routine: its only scratch, the per-block
// partial sums of the energy, is the file-scope device array below.
#include <cmath>
#include <mutex>

#include "ftcj_internal.h"

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_partials[FTCJ_NOALLOC_MAX_PARTIALS];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device, looked up once
// per device with that device current.
int partials_address(double** out) {
    int dev = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return ftcj::fail(FTCJ_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return ftcj::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return FTCJ_OK;
}

struct Metric {
    double m11, m22, m33, m12, m13, m23;
    double four_pi_over_vol, inv_4w2;
};

// W = 2 v conj(rho); partials[d * nblocks + block] = sum over the block of v |rho|^2
__global__ void __launch_bounds__(kNoallocThreads) k_potential_noalloc(
    Metric m, long long ng, const int* __restrict__ gvec, const double2* __restrict__ rho,
    double2* __restrict__ W, double* __restrict__ partials, int nblocks) {
    __shared__ double se[kNoallocThreads];
    const int d = blockIdx.y;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (p < ng) {
        const double n1 = gvec[3 * p], n2 = gvec[3 * p + 1], n3 = gvec[3 * p + 2];
        const double g2 = m.m11 * n1 * n1 + m.m22 * n2 * n2 + m.m33 * n3 * n3 +
                          2.0 * (m.m12 * n1 * n2 + m.m13 * n1 * n3 + m.m23 * n2 * n3);
        const double v = m.four_pi_over_vol * exp(-g2 * m.inv_4w2) / g2;
        const double2 r = rho[(long long)d * ng + p];
        W[(long long)d * ng + p] = make_double2(2.0 * v * r.x, -2.0 * v * r.y);
        e = v * (r.x * r.x + r.y * r.y);
    }
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(long long)d * nblocks + blockIdx.x] = se[0];
}

__global__ void __launch_bounds__(kNoallocThreads) k_energy_noalloc(const double* __restrict__ partials,
                                                                    int nblocks, double* __restrict__ EJ) {
    __shared__ double se[kNoallocThreads];
    const int d = blockIdx.x;
    double e = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) e += partials[(long long)d * nblocks + i];
    se[threadIdx.x] = e;
    __syncthreads();
    for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) se[threadIdx.x] += se[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) EJ[d] = se[0];
}

}  // namespace

extern "C" int ftcj_potential_noalloc(const double A[9], double omega, int ndens, int64_t ng, const int* gvec,
                                      const double* rho, double* W, double* EJ, void* stream) {
    using ftcj::fail;
    if (!A || !EJ || ndens < 1 || ng < 0) return fail(FTCJ_EINVAL, "bad argument");
    if (ng > 0 && (!gvec || !rho || !W)) return fail(FTCJ_EINVAL, "null buffer");
    if (!(omega > 0.0) || !std::isfinite(omega)) return fail(FTCJ_EINVAL, "omega must be > 0");
    const long long nblocks = (ng + kNoallocThreads - 1) / kNoallocThreads;
    if ((long long)ndens * nblocks > FTCJ_NOALLOC_MAX_PARTIALS)
        return fail(FTCJ_EINVAL, "ndens * ceil(ng/256) exceeds FTCJ_NOALLOC_MAX_PARTIALS (16384): split the call");
    // reciprocal lattice b_i = 2 pi (a_j x a_k) / det and metric M_ij = b_i . b_j
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 1e-8)) return fail(FTCJ_EINVAL, "singular lattice");
    double B[9];
    for (int i = 0; i < 3; ++i) {
        const double* u = A + 3 * ((i + 1) % 3);
        const double* v = A + 3 * ((i + 2) % 3);
        B[3 * i + 0] = 2.0 * M_PI * (u[1] * v[2] - u[2] * v[1]) / det;
        B[3 * i + 1] = 2.0 * M_PI * (u[2] * v[0] - u[0] * v[2]) / det;
        B[3 * i + 2] = 2.0 * M_PI * (u[0] * v[1] - u[1] * v[0]) / det;
    }
    auto dot = [&](int i, int j) { return B[3 * i] * B[3 * j] + B[3 * i + 1] * B[3 * j + 1] + B[3 * i + 2] * B[3 * j + 2]; };
    Metric m{dot(0, 0), dot(1, 1), dot(2, 2), dot(0, 1), dot(0, 2), dot(1, 2), 4.0 * M_PI / std::fabs(det),
             1.0 / (4.0 * omega * omega)};
    double* partials = nullptr;
    int rc = partials_address(&partials);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (ng == 0) {
        FTCJ_CUDA(cudaMemsetAsync(EJ, 0, sizeof(double) * ndens, s));
        return FTCJ_OK;
    }
    dim3 g((unsigned)nblocks, (unsigned)ndens);
    k_potential_noalloc<<<g, kNoallocThreads, 0, s>>>(m, ng, gvec, reinterpret_cast<const double2*>(rho),
                                                      reinterpret_cast<double2*>(W), partials, (int)nblocks);
    FTCJ_CUDA(cudaGetLastError());
    k_energy_noalloc<<<ndens, kNoallocThreads, 0, s>>>(partials, (int)nblocks, EJ);
    FTCJ_CUDA(cudaGetLastError());
    return FTCJ_OK;
}
