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
#include <type_traits>
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

// Share s of a sharded build: the records sorted by class are cut where the
// running walk cost (per record and point: 38 L + 100 FP32 operations in the
// split form, 4 L + 24 FP64 operations in the FP64 form, the same constants as
// the rho-walk schedule) first reaches s / S of the total, so that the shares
// take nearly equal walk time on equal GPUs.
void shard_bounds(const int64_t* class_counts, int precision, int shard_count, int64_t* bounds) {
    auto cost = [&](int L) { return precision == FTCJ_PREC_SPLIT ? 38.0 * L + 100.0 : 4.0 * L + 24.0; };
    double total = 0.0;
    int64_t n = 0;
    for (int c = 0; c < kNclass; ++c) {
        total += cost(c) * (double)class_counts[c];
        n += class_counts[c];
    }
    bounds[0] = 0;
    for (int s = 1; s < shard_count; ++s) {
        // the first record index whose running cost reaches s / S of the total
        const double target = total * s / shard_count;
        double acc = 0.0;
        int64_t start = 0, b = n;
        for (int c = 0; c < kNclass; ++c) {
            const double w = cost(c), here = w * (double)class_counts[c];
            if (acc + here >= target) {
                b = start + (int64_t)std::ceil((target - acc) / w - 1e-9);
                break;
            }
            acc += here;
            start += class_counts[c];
        }
        bounds[s] = std::min(std::max(b, bounds[s - 1]), n);
    }
    bounds[shard_count] = n;
}

// Keeps only this plan's share of the class-sorted records (a contiguous
// range): the per-record arrays are cut to it, the class boundaries and the
// ordered-pair count follow.
int keep_record_share(ftcj_plan* P) {
    if (P->shard_count <= 1) return FTCJ_OK;
    int64_t counts[kNclass];
    for (int c = 0; c < kNclass; ++c) counts[c] = P->class_start[c + 1] - P->class_start[c];
    std::vector<int64_t> b((size_t)P->shard_count + 1);
    shard_bounds(counts, P->precision, P->shard_count, b.data());
    const long long first = b[P->shard_index], count = b[P->shard_index + 1] - first;
    std::vector<PairDev> pr((size_t)count);
    if (count > 0)
        FTCJ_CUDA(cudaMemcpy(pr.data(), P->d_pairs + first, sizeof(PairDev) * pr.size(), cudaMemcpyDeviceToHost));
    auto cut = [&](auto** ptr, size_t elem) -> int {
        void* fresh = nullptr;
        FTCJ_CUDA(cudaMalloc(&fresh, elem * (size_t)std::max<long long>(count, 1)));
        if (count > 0) {
            cudaError_t e = cudaMemcpy(fresh, reinterpret_cast<char*>(*ptr) + elem * (size_t)first,
                                       elem * (size_t)count, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) {
                cudaFree(fresh);
                return cuda_fail(e, "record share copy");
            }
        }
        cudaFree(*ptr);
        *ptr = static_cast<std::remove_reference_t<decltype(**ptr)>*>(fresh);
        return FTCJ_OK;
    };
    int rc = cut(&P->d_pairs, sizeof(PairDev));
    if (!rc) rc = cut(&P->d_walk, sizeof(PairWalk));
    if (rc) return rc;
    for (int c = 0; c <= kNclass; ++c)
        P->class_start[c] = std::min<int64_t>(std::max<int64_t>(P->class_start[c] - first, 0), count);
    P->npairs = count;
    P->npairs_ordered = 0;
    for (const PairDev& r : pr)
        P->npairs_ordered += (int64_t)(P->groups[r.ga].mem1 - P->groups[r.ga].mem0) *
                             (P->groups[r.gb].mem1 - P->groups[r.gb].mem0) * r.weight;
    return FTCJ_OK;
}

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
