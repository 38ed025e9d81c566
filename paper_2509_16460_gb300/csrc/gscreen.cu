// Per-pair G cutoffs (Sec. 2.5): after k_pair_gcut has given every pair
// record its own radius, the records of each class are reordered by
// decreasing radius, so that a walk tile (128 consecutive records of one
// class) holds records of similar radius, and each tile walks only the G
// points inside the largest radius of its records.  The reorder permutes the
// per-record arrays (records, walk constants, map offsets, radii); the maps
// themselves stay where they are.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "ftcj_internal.h"

namespace ftcj {
namespace {

template <class T>
__global__ void k_gather(const T* __restrict__ src, const int* __restrict__ perm, long long n, T* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

template <class T>
int permute(ftcj_plan* P, T** ptr, const int* d_perm, long long n) {
    T* fresh = nullptr;
    FTCJ_CUDA(cudaMalloc(&fresh, sizeof(T) * (size_t)n));
    k_gather<<<(unsigned)((n + 255) / 256), 256>>>(*ptr, d_perm, n, fresh);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(fresh);
        return cuda_fail(e, "record permutation");
    }
    cudaFree(*ptr);
    *ptr = fresh;
    return FTCJ_OK;
}

}  // namespace

int apply_pair_cutoffs(ftcj_plan* P) {
    const long long n = P->npairs;
    if (n == 0 || !P->d_rec_gcut) return FTCJ_OK;
    std::vector<float> g((size_t)n);
    std::vector<PairDev> pr((size_t)n);
    FTCJ_CUDA(cudaMemcpy(g.data(), P->d_rec_gcut, sizeof(float) * g.size(), cudaMemcpyDeviceToHost));
    FTCJ_CUDA(cudaMemcpy(pr.data(), P->d_pairs, sizeof(PairDev) * pr.size(), cudaMemcpyDeviceToHost));
    // new position -> old record, by decreasing radius within each class (stable)
    std::vector<int> perm((size_t)n);
    std::iota(perm.begin(), perm.end(), 0);
    for (int c = 0; c < kNclass; ++c)
        std::stable_sort(perm.begin() + P->class_start[c], perm.begin() + P->class_start[c + 1],
                         [&](int a, int b) { return g[a] > g[b]; });
    int* d_perm = nullptr;
    FTCJ_CUDA(cudaMalloc(&d_perm, sizeof(int) * perm.size()));
    cudaError_t e = cudaMemcpy(d_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice);
    int rc = e == cudaSuccess ? FTCJ_OK : cuda_fail(e, "record permutation upload");
    if (!rc) rc = permute(P, &P->d_pairs, d_perm, n);
    if (!rc) rc = permute(P, &P->d_walk, d_perm, n);
    if (!rc) rc = permute(P, &P->d_map_off, d_perm, n);
    if (!rc) rc = permute(P, &P->d_rec_gcut, d_perm, n);
    cudaFree(d_perm);
    if (rc) return rc;
    // squared radii of the half-sphere points, ascending, to count points inside a radius
    std::vector<double> g2((size_t)P->ng_half);
    for (int64_t j = 0; j < P->ng_half; ++j) {
        const double v[3] = {(double)P->gvec[3 * j], (double)P->gvec[3 * j + 1], (double)P->gvec[3 * j + 2]};
        double q = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) q += v[a] * P->M[3 * a + b] * v[b];
        g2[j] = q;
    }
    std::sort(g2.begin(), g2.end());
    auto inside = [&](double r) { return (int64_t)(std::lower_bound(g2.begin(), g2.end(), r * r) - g2.begin()); };
    P->units_screened = 0;
    for (long long i = 0; i < n; ++i) {
        const int o = perm[i];
        P->units_screened += (int64_t)pr[o].weight * 2 * inside(g[o]);
    }
    // each tile walks the radius of its first (largest) record
    P->units_walked = 0;
    P->tile_npts.assign(P->tiles.size(), 0);
    for (size_t t = 0; t < P->tiles.size(); ++t) {
        Tile& tl = P->tiles[t];
        const float r = g[perm[tl.first]];
        tl.gcut2 = r * r;
        const int64_t pts = inside(r);
        P->tile_npts[t] = pts;
        for (int k = 0; k < tl.count; ++k) P->units_walked += (int64_t)pr[perm[tl.first + k]].weight * 2 * pts;
    }
    FTCJ_CUDA(cudaMemcpy(P->d_tiles, P->tiles.data(), sizeof(Tile) * P->tiles.size(), cudaMemcpyHostToDevice));
    return FTCJ_OK;
}

}  // namespace ftcj
