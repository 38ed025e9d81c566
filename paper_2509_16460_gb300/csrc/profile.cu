// Measurement support: per-phase CUDA-event timing of the build, the count
// of kernel launches per batch, and an FMA throughput probe that gives the
// ALU roofline denominators on the GPU the library runs on.
#include <vector>

#include "ftcj_internal.h"

namespace ftcj {

void release_profiling(ftcj_plan* P) {
    for (cudaEvent_t e : P->prof_events)
        if (e) cudaEventDestroy(e);
    P->prof_events.clear();
    P->prof_max = P->prof_used = 0;
    P->prof_launches = 0;
}

int64_t launches_per_batch(const ftcj_plan* P) {
    int axes = 0;
    for (int a = 0; a < 3; ++a) axes += P->km[a] > 1;
    int64_t fold = fused_fold_supported(P) ? 1 : (axes > 0 ? axes : 1);  // fused, stages, or a copy
    int64_t n = 0;
    n += fold;                                         // a2
    n += P->npairs > 0 ? 1 : 0;                        // a3
    n += (P->ng_half > 0 && !P->tiles.empty())
             ? (P->tc ? tc_rho_launches(P, P->max_dens) : (P->rho_hi_tiles > 0 ? 2 : 1))
             : 0;  // a4
    n += P->ng_half > 0 ? 2 : 0;                       // a5: reduce + energy
    n += (P->ng_half > 0 && !P->tiles.empty())
             ? (P->tc_j ? tc_j_launches(P, P->max_dens) : (P->precision == FTCJ_PREC_SPLIT ? split_j_launches(P) : 1))
             : 0;  // a6
    n += P->npairs > 0 ? 1 : 0;                        // a7
    n += fold;                                         // a8
    n += gpw_launches(P, P->max_dens);                 // the DD records' GPW route (classified plans)
    return n;
}

namespace {

// 8 independent FMA chains per thread; the result is only stored when it
// takes an impossible value, so nothing is optimised away.
template <class T>
__global__ void k_fma_probe(T* out, int iters, T b, T c) {
    T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = fma(a0, b, c);
            a1 = fma(a1, b, c);
            a2 = fma(a2, b, c);
            a3 = fma(a3, b, c);
            a4 = fma(a4, b, c);
            a5 = fma(a5, b, c);
            a6 = fma(a6, b, c);
            a7 = fma(a7, b, c);
        }
    }
    T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == (T)-1.2345) out[0] = s;
}

}  // namespace
}  // namespace ftcj

using namespace ftcj;

extern "C" {

int ftcj_profile_enable(ftcj_plan* P, int max_batches) {
    if (!P || max_batches < 0) return fail(FTCJ_EINVAL, "bad argument");
    release_profiling(P);
    if (max_batches == 0) return FTCJ_OK;
    P->prof_events.assign((size_t)max_batches * kProfEvents, nullptr);
    for (auto& e : P->prof_events) FTCJ_CUDA(cudaEventCreate(&e));
    P->prof_max = max_batches;
    return FTCJ_OK;
}

int ftcj_profile_read(ftcj_plan* P, double ms[FTCJ_NPHASE], int* batches, int64_t* launches) {
    if (!P || !ms) return fail(FTCJ_EINVAL, "bad argument");
    for (int i = 0; i < FTCJ_NPHASE; ++i) ms[i] = 0.0;
    for (int b = 0; b < P->prof_used; ++b) {
        cudaEvent_t* ev = P->prof_events.data() + (size_t)b * kProfEvents;
        FTCJ_CUDA(cudaEventSynchronize(ev[7]));
        for (int i = 0; i < FTCJ_NPHASE; ++i) {
            // phases 0..6 between consecutive bounds; 7 and 8 from their own pairs
            const int e0 = i < 7 ? i : 8 + 2 * (i - 7), e1 = i < 7 ? i + 1 : e0 + 1;
            float t = 0.f;
            FTCJ_CUDA(cudaEventElapsedTime(&t, ev[e0], ev[e1]));
            ms[i] += t;
        }
    }
    if (batches) *batches = P->prof_used;
    if (launches) *launches = P->prof_launches;
    P->prof_used = 0;
    P->prof_launches = 0;
    return FTCJ_OK;
}

int ftcj_launches_per_batch(const ftcj_plan* P, int nd, int64_t* launches) {
    if (!P || !launches || nd < 1) return fail(FTCJ_EINVAL, "bad argument");
    *launches = launches_per_batch(P);
    return FTCJ_OK;
}

int ftcj_probe_fma_peak(int precision, double* flops_per_s, void* stream) {
    if (!flops_per_s || (precision != 0 && precision != 1)) return fail(FTCJ_EINVAL, "bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    void* out = nullptr;
    FTCJ_CUDA(cudaMalloc(&out, 16));
    cudaEvent_t e0, e1;
    FTCJ_CUDA(cudaEventCreate(&e0));
    FTCJ_CUDA(cudaEventCreate(&e1));
    const int threads = 256, blocks = sms * 8;
    const int iters = precision == 0 ? 400 : 20000;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        FTCJ_CUDA(cudaEventRecord(e0, s));
        if (precision == 0)
            k_fma_probe<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
        else
            k_fma_probe<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        FTCJ_CUDA(cudaGetLastError());
        FTCJ_CUDA(cudaEventRecord(e1, s));
        FTCJ_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        FTCJ_CUDA(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0 && t < best) best = t;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    double flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)threads * (double)blocks;
    *flops_per_s = flops / (best * 1e-3);
    return FTCJ_OK;
}

}  // extern "C"
