// Step a1 on the device: screen candidate primitive pairs (group a in the home
// cell, group b in cell L) by their overlap bound (and, in a classified plan,
// by density class: compact or DD, Sec. 2.6), keep one record per mirror
// couple (a0,bL) <-> (b0,a-L), and sort the survivors stably by the pair
// class L = l_a + l_b (counting sort by tiles).  The epilogue computes each
// record's Gaussian-product data (Eqs. GPT) and the constants of the G walk.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ftcj_internal.h"

namespace ftcj {
namespace {


// ---- block-wide exclusive scan ------------------------------------------
__device__ long long block_scan_excl(long long v, long long* s_tot, long long* s_warp) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int nw = (blockDim.x + 31) >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = (lane < nw) ? s_warp[lane] : 0;
        long long s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) s_warp[lane] = s - t;
        if (lane == nw - 1) *s_tot = s;
    }
    __syncthreads();
    long long r = s_warp[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_block(const long long* __restrict__ in, long long* __restrict__ out,
                             long long* __restrict__ bsum, long long n) {
    __shared__ long long s_tot, s_warp[32];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = i < n ? in[i] : 0;
    long long e = block_scan_excl(v, &s_tot, s_warp);
    if (i < n) out[i] = e;
    if (threadIdx.x == 0) bsum[blockIdx.x] = s_tot;
}

__global__ void k_scan_bsum(long long* bsum, long long nb) {
    __shared__ long long s_tot, s_warp[32];
    long long carry = 0;
    for (long long base = 0; base < nb; base += blockDim.x) {
        long long i = base + threadIdx.x;
        long long v = i < nb ? bsum[i] : 0;
        long long e = block_scan_excl(v, &s_tot, s_warp);
        if (i < nb) bsum[i] = e + carry;
        carry += s_tot;
        __syncthreads();
    }
}

__global__ void k_scan_add(long long* out, const long long* __restrict__ bsum, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// ---- candidate boxes ----------------------------------------------------
__global__ void k_screen_count(const GroupDev* __restrict__ G, int ng, double thr, long long* __restrict__ cnt,
                               int* __restrict__ lim, CellConst cc) {
    int ga = blockIdx.y;
    int gb = blockIdx.x * blockDim.x + threadIdx.x;
    if (gb >= ng) return;
    long long gp = (long long)ga * ng + gb;
    long long n = 0;
    int l0 = 0, l1 = 0, l2 = 0;
    if (gb >= ga) {
        double a = G[ga].alpha, b = G[gb].alpha;
        double p = a + b, mu = a * b / p;
        double s0 = pow(2.0 * sqrt(a * b) / p, 1.5);
        if (s0 > thr) {
            double dx = G[ga].x - G[gb].x, dy = G[ga].y - G[gb].y, dz = G[ga].z - G[gb].z;
            double dab = sqrt(dx * dx + dy * dy + dz * dz);
            double rmax = sqrt(log(s0 / thr) / mu);
            l0 = (int)ceil((dab + rmax) * cc.bn[0] / (2.0 * M_PI)) + 1;
            l1 = (int)ceil((dab + rmax) * cc.bn[1] / (2.0 * M_PI)) + 1;
            l2 = (int)ceil((dab + rmax) * cc.bn[2] / (2.0 * M_PI)) + 1;
            n = (long long)(2 * l0 + 1) * (2 * l1 + 1) * (2 * l2 + 1);
        }
    }
    cnt[gp] = n;
    lim[3 * gp + 0] = l0;
    lim[3 * gp + 1] = l1;
    lim[3 * gp + 2] = l2;
}

struct Cand {
    int ga, gb, L0, L1, L2;
};

// candidate index -> (group pair, L) via the exclusive offsets of the boxes
__device__ __forceinline__ Cand decode(const long long* __restrict__ off, const int* __restrict__ lim, int ng,
                                       long long c) {
    long long lo = 0, hi = (long long)ng * ng;  // last index with off <= c (a non-empty box)
    while (hi - lo > 1) {
        long long mid = (lo + hi) >> 1;
        if (off[mid] <= c) lo = mid;
        else hi = mid;
    }
    long long gp = lo;
    long long loc = c - off[gp];
    int l0 = lim[3 * gp], l1 = lim[3 * gp + 1], l2 = lim[3 * gp + 2];
    int w1 = 2 * l1 + 1, w2 = 2 * l2 + 1;
    Cand r;
    r.ga = (int)(gp / ng);
    r.gb = (int)(gp % ng);
    r.L0 = (int)(loc / ((long long)w1 * w2)) - l0;
    r.L1 = (int)((loc / w2) % w1) - l1;
    r.L2 = (int)(loc % w2) - l2;
    return r;
}

__global__ void k_screen_eval(const GroupDev* __restrict__ G, int ng, double thr, const long long* __restrict__ off,
                              const int* __restrict__ lim, long long C, unsigned char* __restrict__ flag,
                              unsigned char* __restrict__ key, CellConst cc, double acut, int filter) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    Cand q = decode(off, lim, ng, c);
    GroupDev A = G[q.ga];
    GroupDev B = G[q.gb];
    double a = A.alpha, b = B.alpha, p = a + b;
    double AB[3] = {A.x - B.x, A.y - B.y, A.z - B.z};
    double r2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double R = AB[x] - (q.L0 * cc.A[x] + q.L1 * cc.A[3 + x] + q.L2 * cc.A[6 + x]);
        r2 += R * R;
    }
    double s = pow(2.0 * sqrt(a * b) / p, 1.5) * exp(-a * b / p * r2);
    bool ok = s > thr;
    if (q.ga == q.gb) {  // keep one of (a0,aL) and (a0,a-L)
        bool nonneg = q.L0 > 0 || (q.L0 == 0 && (q.L1 > 0 || (q.L1 == 0 && q.L2 >= 0)));
        ok = ok && nonneg;
    }
    if (filter) {  // density classes (Sec. 2.6): DD when both exponents lie below alpha_cut
        const bool dd = a < acut && b < acut;
        ok = ok && (filter == 2 ? dd : !dd);
    }
    flag[c] = ok ? 1 : 0;
    key[c] = (unsigned char)(A.lmax + B.lmax);
}

__global__ void k_tile_count(const unsigned char* __restrict__ flag, const unsigned char* __restrict__ key,
                             long long C, long long ntiles, long long* __restrict__ tc) {
    __shared__ int cnt[kNclass];
    if (threadIdx.x < kNclass) cnt[threadIdx.x] = 0;
    __syncthreads();
    long long c = (long long)blockIdx.x * kSortTile + threadIdx.x;
    if (c < C && flag[c]) atomicAdd(&cnt[key[c]], 1);
    __syncthreads();
    if (threadIdx.x < kNclass) tc[(long long)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// stable scatter: inside a tile the rank of a survivor among the same class
// is its block-wide exclusive prefix, so candidate order is preserved
__global__ void k_tile_scatter(const unsigned char* __restrict__ flag, const unsigned char* __restrict__ key,
                               long long C, long long ntiles, const long long* __restrict__ toff,
                               long long* __restrict__ order) {
    __shared__ long long s_tot, s_warp[32];
    long long c = (long long)blockIdx.x * kSortTile + threadIdx.x;
    int f = (c < C) ? flag[c] : 0;
    int k = (c < C) ? key[c] : -1;
    for (int kk = 0; kk < kNclass; ++kk) {
        long long v = (f && k == kk) ? 1 : 0;
        long long e = block_scan_excl(v, &s_tot, s_warp);
        if (v) order[toff[(long long)kk * ntiles + blockIdx.x] + e] = c;
    }
}

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__global__ void k_pair_setup(const GroupDev* __restrict__ G, const int* __restrict__ nmem, int ng,
                             const long long* __restrict__ off, const int* __restrict__ lim,
                             const long long* __restrict__ order, long long npairs, PairDev* __restrict__ pairs,
                             PairWalk* __restrict__ walk, unsigned long long* __restrict__ units, CellConst cc) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    Cand q = decode(off, lim, ng, order[i]);
    GroupDev A = G[q.ga];
    GroupDev B = G[q.gb];
    double a = A.alpha, b = B.alpha, p = a + b, mu = a * b / p;
    double Av[3] = {A.x, A.y, A.z};
    double Bv[3] = {B.x, B.y, B.z};
    PairDev r;
    r.ga = q.ga;
    r.gb = q.gb;
    r.L[0] = q.L0;
    r.L[1] = q.L1;
    r.L[2] = q.L2;
    r.cell = (wrapi(q.L0, cc.km[0]) * cc.km[1] + wrapi(q.L1, cc.km[1])) * cc.km[2] + wrapi(q.L2, cc.km[2]);
    r.mcell = (wrapi(-q.L0, cc.km[0]) * cc.km[1] + wrapi(-q.L1, cc.km[1])) * cc.km[2] + wrapi(-q.L2, cc.km[2]);
    bool self = (q.ga == q.gb) && q.L0 == 0 && q.L1 == 0 && q.L2 == 0;
    r.weight = self ? 1 : 2;
    r.cls = A.lmax + B.lmax;
    r.pad = 0;
    double r2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double Bs = Bv[x] + q.L0 * cc.A[x] + q.L1 * cc.A[3 + x] + q.L2 * cc.A[6 + x];
        r.P[x] = (a * Av[x] + b * Bs) / p;
        double d = Av[x] - Bs;
        r2 += d * d;
    }
    r.p = p;
    r.K = exp(-mu * r2) * pow(M_PI / p, 1.5);
    pairs[i] = r;

    PairWalk w;
    double c = 0.25 / p;
    w.c = c;
    double f[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double fj = cc.Bt[3 * j] * r.P[0] + cc.Bt[3 * j + 1] * r.P[1] + cc.Bt[3 * j + 2] * r.P[2];
        f[j] = fj - rint(fj);
    }
    w.f1 = f[0];
    w.f2 = f[1];
    w.f3 = f[2];
    w.q1 = exp(-2.0 * c * cc.M6[0]);
    w.q2 = exp(-2.0 * c * cc.M6[1]);
    w.q3 = exp(-2.0 * c * cc.M6[2]);
    w.x12 = exp(-2.0 * c * cc.M6[3]);
    w.y12 = exp(2.0 * c * cc.M6[3]);
    w.x13 = exp(-2.0 * c * cc.M6[4]);
    w.y13 = exp(2.0 * c * cc.M6[4]);
    w.x23 = exp(-2.0 * c * cc.M6[5]);
    w.y23 = exp(2.0 * c * cc.M6[5]);
    double s, co;
    sincospi(2.0 * f[0], &s, &co);
    w.e1r = co;
    w.e1i = -s;
    sincospi(2.0 * f[1], &s, &co);
    w.e2r = co;
    w.e2i = -s;
    sincospi(2.0 * f[2], &s, &co);
    w.e3r = co;
    w.e3i = -s;
    w.pad = 0.0;
    walk[i] = w;
    units[i] = (unsigned long long)nmem[q.ga] * (unsigned long long)nmem[q.gb] * (unsigned long long)r.weight;
}

__global__ void k_sum_u64(const unsigned long long* __restrict__ v, long long n, unsigned long long* out) {
    __shared__ unsigned long long s[256];
    unsigned long long acc = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, s[0]);
}

struct Scratch {
    void* p[16] = {};
    int n = 0;
    ~Scratch() {
        for (int i = 0; i < n; ++i)
            if (p[i]) cudaFree(p[i]);
    }
    template <class T>
    cudaError_t get(T** ptr, size_t count) {
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)ptr, sizeof(T) * count);
        p[n++] = *ptr;
        return e;
    }
};

}  // namespace

// exclusive scan of n int64 values on the device; the total comes back to the host
static int exclusive_scan(const long long* in, long long* out, long long n, long long* total) {
    if (n <= 0) {
        *total = 0;
        return FTCJ_OK;
    }
    long long nb = (n + 1023) / 1024;
    Scratch s;
    long long* bsum = nullptr;
    FTCJ_CUDA(s.get(&bsum, (size_t)nb));
    k_scan_block<<<(unsigned)nb, 1024>>>(in, out, bsum, n);
    FTCJ_CUDA(cudaGetLastError());
    k_scan_bsum<<<1, 1024>>>(bsum, nb);
    FTCJ_CUDA(cudaGetLastError());
    k_scan_add<<<(unsigned)nb, 1024>>>(out, bsum, n);
    FTCJ_CUDA(cudaGetLastError());
    long long last_in = 0, last_out = 0;
    FTCJ_CUDA(cudaMemcpy(&last_in, in + n - 1, sizeof(long long), cudaMemcpyDeviceToHost));
    FTCJ_CUDA(cudaMemcpy(&last_out, out + n - 1, sizeof(long long), cudaMemcpyDeviceToHost));
    *total = last_in + last_out;
    return FTCJ_OK;
}

int screen_and_sort(ftcj_plan* P) {
    const CellConst cc = P->cc;

    int ng = P->ngroup;
    long long ngp = (long long)ng * ng;
    double thr = P->params.pair_thresh;
    Scratch s;
    long long *cnt = nullptr, *off = nullptr;
    int* lim = nullptr;
    int* nmem = nullptr;
    FTCJ_CUDA(s.get(&cnt, (size_t)ngp));
    FTCJ_CUDA(s.get(&off, (size_t)ngp));
    FTCJ_CUDA(s.get(&lim, (size_t)ngp * 3));
    FTCJ_CUDA(s.get(&nmem, (size_t)ng));
    std::vector<int> hn(ng);
    for (int g = 0; g < ng; ++g) hn[g] = P->groups[g].mem1 - P->groups[g].mem0;
    FTCJ_CUDA(cudaMemcpy(nmem, hn.data(), sizeof(int) * ng, cudaMemcpyHostToDevice));

    if (ng > 65535) return fail(FTCJ_EUNSUPPORTED, "more than 65535 primitive groups");
    dim3 gc((ng + 127) / 128, ng);
    k_screen_count<<<gc, 128>>>(P->d_groups, ng, thr, cnt, lim, cc);
    FTCJ_CUDA(cudaGetLastError());
    long long C = 0;
    int rc = exclusive_scan(cnt, off, ngp, &C);
    if (rc) return rc;

    long long ntiles = std::max<long long>(1, (C + kSortTile - 1) / kSortTile);
    unsigned char *flag = nullptr, *key = nullptr;
    long long *tc = nullptr, *toff = nullptr;
    FTCJ_CUDA(s.get(&flag, (size_t)std::max<long long>(C, 1)));
    FTCJ_CUDA(s.get(&key, (size_t)std::max<long long>(C, 1)));
    FTCJ_CUDA(s.get(&tc, (size_t)(ntiles * kNclass)));
    FTCJ_CUDA(s.get(&toff, (size_t)(ntiles * kNclass)));
    if (C > 0) {
        k_screen_eval<<<(unsigned)((C + 255) / 256), 256>>>(P->d_groups, ng, thr, off, lim, C, flag, key, cc,
                                                             P->alpha_cut, P->rec_filter);
        FTCJ_CUDA(cudaGetLastError());
    }
    k_tile_count<<<(unsigned)ntiles, kSortTile>>>(flag, key, C, ntiles, tc);
    FTCJ_CUDA(cudaGetLastError());
    long long npairs = 0;
    rc = exclusive_scan(tc, toff, ntiles * kNclass, &npairs);
    if (rc) return rc;
    P->npairs = npairs;
    // class boundaries: the offset of each class's first tile
    std::vector<long long> starts(kNclass);
    for (int k = 0; k < kNclass; ++k)
        FTCJ_CUDA(cudaMemcpy(&starts[k], toff + (long long)k * ntiles, sizeof(long long), cudaMemcpyDeviceToHost));
    for (int k = 0; k < kNclass; ++k) P->class_start[k] = starts[k];
    P->class_start[kNclass] = npairs;

    long long* order = nullptr;
    FTCJ_CUDA(s.get(&order, (size_t)std::max<long long>(npairs, 1)));
    k_tile_scatter<<<(unsigned)ntiles, kSortTile>>>(flag, key, C, ntiles, toff, order);
    FTCJ_CUDA(cudaGetLastError());

    FTCJ_CUDA(cudaMalloc(&P->d_pairs, sizeof(PairDev) * (size_t)std::max<long long>(npairs, 1)));
    P->device_bytes += sizeof(PairDev) * (size_t)std::max<long long>(npairs, 1);
    FTCJ_CUDA(cudaMalloc(&P->d_walk, sizeof(PairWalk) * (size_t)std::max<long long>(npairs, 1)));
    P->device_bytes += sizeof(PairWalk) * (size_t)std::max<long long>(npairs, 1);
    unsigned long long *units = nullptr, *utot = nullptr;
    FTCJ_CUDA(s.get(&units, (size_t)std::max<long long>(npairs, 1)));
    FTCJ_CUDA(s.get(&utot, 1));
    FTCJ_CUDA(cudaMemset(utot, 0, sizeof(unsigned long long)));
    if (npairs > 0) {
        k_pair_setup<<<(unsigned)((npairs + 255) / 256), 256>>>(P->d_groups, nmem, ng, off, lim, order, npairs,
                                                                 P->d_pairs, P->d_walk, units, cc);
        FTCJ_CUDA(cudaGetLastError());
        k_sum_u64<<<256, 256>>>(units, npairs, utot);
        FTCJ_CUDA(cudaGetLastError());
    }
    unsigned long long h = 0;
    FTCJ_CUDA(cudaMemcpy(&h, utot, sizeof(h), cudaMemcpyDeviceToHost));
    P->npairs_ordered = (int64_t)h;
    FTCJ_CUDA(cudaDeviceSynchronize());
    return FTCJ_OK;
}

}  // namespace ftcj
