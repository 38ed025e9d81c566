// Plan construction for the long-range Coulomb build: input validation,
// reciprocal lattice and metric, primitive groups (several shells sharing one
// primitive are processed together, Sec. 2.4 "multishell"), the walk over the
// half G sphere as lines along b_1 (Sec. 2.5, Eq. "G-space root finding"),
// device allocation, and the device-side pair screening.
#include <algorithm>
#include <queue>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "ftcj_internal.h"

namespace ftcj {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FTCJ_ECUDA;
}

// Raises the kernel's dynamic shared-memory limit to what the device allows
// beside its static shared memory (the attribute is per kernel and global, so
// it is set to the maximum once rather than to one plan's need).
int allow_dynamic_smem(const void* func, size_t need) {
    int dev = 0, optin = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    FTCJ_CUDA(cudaFuncGetAttributes(&fa, func));
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (need > room) return fail(FTCJ_EUNSUPPORTED, "shared memory of a walk chunk above the device limit");
    FTCJ_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room));
    return FTCJ_OK;
}

namespace {

bool finite(double x) { return std::isfinite(x); }

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// |G|^2 = n^T M n for the metric M_ij = b_i . b_j
double qform(const double* M, long n1, long n2, long n3) {
    double n[3] = {(double)n1, (double)n2, (double)n3};
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += n[i] * M[3 * i + j] * n[j];
    return s;
}

// n1 range of the line (n2, n3) inside |G|^2 < gc2: the roots of
// M11 n^2 + 2 (M12 n2 + M13 n3) n + Q(0,n2,n3) - gc2 = 0, refined by exact tests.
bool line_range(const double* M, double gc2, int n2, int n3, int* lo, int* hi) {
    double M11 = M[0];
    double beta = M[1] * n2 + M[2] * n3;
    double c0 = qform(M, 0, n2, n3) - gc2;
    double disc = beta * beta - M11 * c0;
    double x0 = -beta / M11;
    double h = disc > 0 ? std::sqrt(disc) / M11 : 0.0;
    long a = (long)std::ceil(x0 - h) - 1;
    long b = (long)std::floor(x0 + h) + 1;
    while (a <= b && !(qform(M, a, n2, n3) < gc2)) ++a;
    while (b >= a && !(qform(M, b, n2, n3) < gc2)) --b;
    if (a > b) return false;
    while (qform(M, a - 1, n2, n3) < gc2) --a;
    while (qform(M, b + 1, n2, n3) < gc2) ++b;
    *lo = (int)a;
    *hi = (int)b;
    return true;
}

int build_walk(ftcj_plan* P) {
    const double* M = P->M;
    double gc2 = P->gcut * P->gcut;
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        double an = std::sqrt(dot3(P->A + 3 * i, P->A + 3 * i));
        lim[i] = (int)std::floor(P->gcut * an / (2.0 * M_PI)) + 1;
    }
    P->lines.clear();
    P->gvec.clear();
    struct Raw {
        int n2, n3, lo, hi;
    };
    std::vector<Raw> raw;
    std::vector<int> op;
    // planes n3 = 0..last non-empty
    int n3_last = -1;
    for (int n3 = 0; n3 <= lim[2]; ++n3) {
        bool any = false;
        for (int n2 = -lim[1]; n2 <= lim[1] && !any; ++n2) {
            if (n3 == 0 && n2 < 0) continue;
            int lo, hi;
            if (line_range(M, gc2, n2, n3, &lo, &hi)) {
                if (n3 == 0 && n2 == 0) lo = std::max(lo, 1);
                if (lo <= hi) any = true;
            }
        }
        if (any) n3_last = n3;
    }
    for (int n3 = 0; n3 <= n3_last; ++n3) {
        int pos_last = 0, neg_last = 0;
        std::map<int, std::pair<int, int>> rng;
        for (int n2 = -lim[1]; n2 <= lim[1]; ++n2) {
            if (n3 == 0 && n2 < 0) continue;
            int lo, hi;
            if (!line_range(M, gc2, n2, n3, &lo, &hi)) continue;
            if (n3 == 0 && n2 == 0) lo = std::max(lo, 1);
            if (lo > hi) continue;
            rng[n2] = {lo, hi};
            if (n2 >= 0) pos_last = std::max(pos_last, n2);
            else neg_last = std::min(neg_last, n2);
        }
        for (int n2 = 0; n2 <= pos_last; ++n2) {
            auto it = rng.find(n2);
            int lo = 1, hi = 0;
            if (it != rng.end()) {
                lo = it->second.first;
                hi = it->second.second;
            }
            raw.push_back({n2, n3, lo, hi});
            op.push_back(n2 == 0 ? (n3 == 0 ? OP_FIRST : OP_N3) : OP_N2F);
        }
        for (int n2 = -1; n2 >= neg_last && n3 > 0; --n2) {
            auto it = rng.find(n2);
            int lo = 1, hi = 0;
            if (it != rng.end()) {
                lo = it->second.first;
                hi = it->second.second;
            }
            raw.push_back({n2, n3, lo, hi});
            op.push_back(n2 == -1 ? OP_NEGSTART : OP_N2B);
        }
    }
    // chunks and point order
    P->chunks.clear();
    int pt = 0, cur = 0, l0 = 0, p0 = 0;
    int n1min = 0, n1max = 0;
    for (size_t i = 0; i < raw.size(); ++i) {
        int npts = raw[i].hi >= raw[i].lo ? raw[i].hi - raw[i].lo + 1 : 0;
        if (npts > P->chunk_max) return fail(FTCJ_EUNSUPPORTED, "a G line is longer than the walk chunk");
        if (cur > 0 && cur + npts > P->chunk_max) {
            P->chunks.push_back({l0, (int)i, p0, pt});
            l0 = (int)i;
            p0 = pt;
            cur = 0;
        }
        int o = (i == (size_t)l0) ? OP_FIRST : op[i];
        const double qb = M[1] * raw[i].n2 + M[2] * raw[i].n3;
        P->lines.push_back({raw[i].n2, raw[i].n3, raw[i].lo, raw[i].hi, o, pt, (float)M[0], (float)qb,
                            (float)qform(M, 0, raw[i].n2, raw[i].n3)});
        if (npts > 0) {
            for (int n1 = std::max(raw[i].lo, 0); n1 <= raw[i].hi; ++n1) {
                P->gvec.push_back(n1);
                P->gvec.push_back(raw[i].n2);
                P->gvec.push_back(raw[i].n3);
            }
            for (int n1 = std::min(raw[i].hi, -1); n1 >= raw[i].lo; --n1) {
                P->gvec.push_back(n1);
                P->gvec.push_back(raw[i].n2);
                P->gvec.push_back(raw[i].n3);
            }
            n1min = std::min(n1min, raw[i].lo);
            n1max = std::max(n1max, raw[i].hi);
        }
        pt += npts;
        cur += npts;
    }
    if (!raw.empty()) P->chunks.push_back({l0, (int)raw.size(), p0, pt});
    P->ng_half = pt;
    P->max_chunk_pts = 0;
    for (auto& c : P->chunks) P->max_chunk_pts = std::max(P->max_chunk_pts, c.p1 - c.p0);
    P->n1_min = n1min;
    P->n1_max = n1max;
    return FTCJ_OK;
}

// Default walk chunk of the split form: the structure-factor block keeps one
// chunk's rho row (16 B per point) in shared memory beside chunk-independent
// staging, so the chunk sets its occupancy.  Take the largest power of two
// (<= 4096 points) that lets three blocks of the one-kernel walk share an SM
// with at least 1024 points; else three blocks of its classes 0-2 part (the
// walk then runs in two launches by class) with at least 512; else two blocks
// of the one-kernel walk.  The walk program is rebuilt for it.
int default_split_chunk(ftcj_plan* P) {
    int dev = 0, per_sm = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int keep = P->max_chunk_pts;
    P->max_chunk_pts = 0;
    const size_t fixed_all = split_rho_smem(P, 0), fixed_low = split_rho_smem(P, 1);
    P->max_chunk_pts = keep;
    struct Try {
        int blocks;
        size_t fixed;
        long long need;
    };
    const Try tries[] = {{3, fixed_all, 1024}, {3, fixed_low, 512}, {2, fixed_all, 512}, {1, fixed_all, 64}};
    int chunk = 256;
    for (const Try& t : tries) {
        const long long room = (long long)per_sm / t.blocks - 1024 - (long long)t.fixed;
        const long long pts = room / 16;
        if (pts >= t.need && pts >= 64) {
            chunk = 64;
            while (chunk * 2 <= std::min<long long>(pts, kChunkMax)) chunk *= 2;
            break;
        }
    }
    if (chunk >= P->chunk_max) return FTCJ_OK;
    P->chunk_max = chunk;
    return build_walk(P);
}

template <class T>
int dalloc(ftcj_plan* P, T** ptr, size_t count) {
    if (count == 0) count = 1;
    size_t bytes = sizeof(T) * count;
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(FTCJ_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                     cudaGetErrorString(e));
    }
    P->device_bytes += bytes;
    return FTCJ_OK;
}

template <class T>
int upload(ftcj_plan* P, T** ptr, const std::vector<T>& v) {
    int rc = dalloc(P, ptr, v.size());
    if (rc) return rc;
    if (!v.empty()) FTCJ_CUDA(cudaMemcpy(*ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return FTCJ_OK;
}

// Longest-processing-time assignment of the rho pass's tiles to its npb
// persistent blocks (each block sums its tiles into its own row, so the
// assignment is fixed at plan time and the sums stay deterministic).  A tile
// walks every point of the chunk, so its cost is set by its class L: per point
// the split form spends about 38L + 100 FP32 operations (polynomial, phase
// product, batch reduction), the FP64 form about 4L + 24 FP64 operations.
// With the split walk in two launches (rho_hi_tiles > 0) the leading tiles of
// classes 3-4 go to blocks [0, npb_hi) and the rest to [npb_hi, npb), each
// group by its own assignment.
int build_rho_schedule(ftcj_plan* P) {
    const int nt = (int)P->tiles.size(), nb = std::max(1, P->npb);
    auto cost = [&](int t) {
        const double L = (double)P->tiles[t].cls;
        const double pts = P->tile_npts.empty() ? 1.0 : (double)P->tile_npts[t] + 1.0;  // radius-limited tiles
        return (P->precision == FTCJ_PREC_SPLIT ? 38.0 * L + 100.0 : 4.0 * L + 24.0) * pts;
    };
    std::vector<std::vector<int>> lists(nb);
    auto assign = [&](int t0, int t1, int b0, int b1) {
        std::vector<int> order;
        for (int t = t0; t < t1; ++t) order.push_back(t);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
        using Slot = std::pair<double, int>;  // (load, block): ties go to the lower block
        std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
        for (int b = b0; b < b1; ++b) heap.push({0.0, b});
        for (int t : order) {
            Slot s = heap.top();
            heap.pop();
            lists[s.second].push_back(t);
            heap.push({s.first + cost(t), s.second});
        }
    };
    if (P->rho_hi_tiles > 0) {
        assign(0, P->rho_hi_tiles, 0, P->npb_hi);
        assign(P->rho_hi_tiles, nt, P->npb_hi, nb);
    } else {
        assign(0, nt, 0, nb);
    }
    std::vector<int> sched;
    sched.reserve((size_t)nb + 1 + nt);
    int off = 0;
    for (int b = 0; b < nb; ++b) {
        sched.push_back(off);
        off += (int)lists[b].size();
    }
    sched.push_back(off);
    for (int b = 0; b < nb; ++b) sched.insert(sched.end(), lists[b].begin(), lists[b].end());
    P->rho_sched = sched;
    if (P->d_sched) {
        cudaFree(P->d_sched);
        P->d_sched = nullptr;
    }
    return upload(P, &P->d_sched, P->rho_sched);
}

void free_device(ftcj_plan* P) {
    void* ptrs[] = {P->d_groups, P->d_members, P->d_pairs, P->d_walk, P->d_lines, P->d_chunks, P->d_tiles,
                    P->d_gvec, P->d_vg, P->d_tw, P->d_Tmat, P->d_D0n, P->d_J0n, P->d_cbuf0, P->d_cbuf1,
                    P->d_Dp, P->d_Jp, P->d_rho_part, P->d_rho, P->d_W, P->d_Epart, P->d_Dk_stage,
                    P->d_Jk_stage, P->d_EJ_stage, P->d_check, P->d_split_init, P->d_split_const, P->d_Jg,
                    P->d_maps, P->d_map_off, P->d_sched, P->d_rec_gcut, P->d_tc_rows, P->d_tc_map,
                    P->d_tc_kappa, P->d_tc_tab, P->d_tc_cl, P->d_tc_err, P->d_tc_wpairs, P->d_tc_winfo,
                    P->d_tc_pos, P->d_tc_jitems, P->d_tc_jpairs, P->d_tc_vs, P->d_tc_ev,
                    P->d_tc_ebw, P->d_tc_clw};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    free_gpw(P);
    if (P->dd) {
        free_device(P->dd);
        delete P->dd;
        P->dd = nullptr;
    }
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->aux) cudaStreamDestroy(P->aux);
}

int create(const ftcj_cell* cell, const ftcj_basis* basis, const int kmesh[3], const ftcj_params* prm,
           ftcj_plan* P) {
    if (!cell || !basis || !kmesh || !prm) return fail(FTCJ_EINVAL, "null argument");
    P->params = *prm;
    // lattice
    for (int i = 0; i < 9; ++i) {
        if (!finite(cell->A[i])) return fail(FTCJ_EINVAL, "non-finite lattice");
        P->A[i] = cell->A[i];
    }
    const double* a = P->A;
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                 a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (!(std::fabs(det) > 1e-8)) return fail(FTCJ_EINVAL, "singular lattice");
    P->vol = std::fabs(det);
    for (int i = 0; i < 3; ++i) {
        const double* u = a + 3 * ((i + 1) % 3);
        const double* v = a + 3 * ((i + 2) % 3);
        P->B[3 * i + 0] = 2.0 * M_PI * (u[1] * v[2] - u[2] * v[1]) / det;
        P->B[3 * i + 1] = 2.0 * M_PI * (u[2] * v[0] - u[0] * v[2]) / det;
        P->B[3 * i + 2] = 2.0 * M_PI * (u[0] * v[1] - u[1] * v[0]) / det;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = dot3(P->B + 3 * i, P->B + 3 * j);
    std::memset(&P->cc, 0, sizeof(P->cc));
    for (int i = 0; i < 9; ++i) {
        P->cc.A[i] = P->A[i];
        P->cc.Bt[i] = P->B[i] / (2.0 * M_PI);
    }
    {
        const double m6[6] = {P->M[0], P->M[4], P->M[8], P->M[1], P->M[2], P->M[5]};
        for (int i = 0; i < 6; ++i) P->cc.M6[i] = m6[i];
        for (int i = 0; i < 3; ++i) P->cc.bn[i] = std::sqrt(P->M[4 * i]);
        P->ortho = m6[3] == 0.0 && m6[4] == 0.0 && m6[5] == 0.0;
    }
    // k mesh
    P->nk = 1;
    for (int i = 0; i < 3; ++i) {
        if (kmesh[i] < 1) return fail(FTCJ_EINVAL, "k-mesh dimensions must be >= 1");
        if (kmesh[i] > 16) return fail(FTCJ_EUNSUPPORTED, "k-mesh dimension above 16");
        P->km[i] = kmesh[i];
        P->cc.km[i] = kmesh[i];
        P->nk *= kmesh[i];
    }
    // parameters
    if (!(prm->omega > 0.0) || !finite(prm->omega)) return fail(FTCJ_EINVAL, "omega must be > 0");
    if (prm->precision != FTCJ_PREC_FP64 && prm->precision != FTCJ_PREC_SPLIT)
        return fail(FTCJ_EUNSUPPORTED, "precision must be FTCJ_PREC_FP64 or FTCJ_PREC_SPLIT");
    P->precision = prm->precision;
    if (!(prm->pair_gcut_eps >= 0.0) || !finite(prm->pair_gcut_eps))
        return fail(FTCJ_EINVAL, "pair_gcut_eps must be a finite number >= 0");
    if (prm->shard_count > 1 && (prm->shard_index < 0 || prm->shard_index >= prm->shard_count))
        return fail(FTCJ_EINVAL, "shard_index must be in [0, shard_count)");
    P->shard_count = std::max(1, prm->shard_count);
    P->shard_index = P->shard_count > 1 ? prm->shard_index : 0;
    if (prm->tc_wait_log2 < 0 || prm->tc_wait_log2 > 40) return fail(FTCJ_EINVAL, "tc_wait_log2 must be 0..40");
    if (prm->contraction != FTCJ_CONTRACT_WALK && prm->contraction != FTCJ_CONTRACT_TC)
        return fail(FTCJ_EINVAL, "contraction must be FTCJ_CONTRACT_WALK or FTCJ_CONTRACT_TC");
    P->tc = prm->contraction == FTCJ_CONTRACT_TC;
    if (P->tc && prm->precision != FTCJ_PREC_SPLIT)
        return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction is part of the split-precision form");
    if (P->tc && prm->pair_gcut_eps > 0.0)
        return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction covers the whole sphere (pair_gcut_eps = 0)");
    if (!(prm->pair_thresh > 0.0 && prm->pair_thresh < 1.0)) return fail(FTCJ_EINVAL, "pair_thresh in (0,1)");
    if (prm->classify != 0 && prm->classify != 1) return fail(FTCJ_EINVAL, "classify must be 0 or 1");
    if (prm->classify) {
        if (P->shard_count > 1)
            return fail(FTCJ_EUNSUPPORTED, "a classified plan (compact/diffuse) is not record-sharded");
        if (!finite(prm->alpha_cut)) return fail(FTCJ_EINVAL, "alpha_cut must be finite");
        if (prm->pair_gcut_eps > 0.0)
            return fail(FTCJ_EUNSUPPORTED, "per-pair cutoffs are derived for the long-range kernel alone; a "
                                           "classified plan walks the whole sphere (pair_gcut_eps = 0)");
        P->alpha_cut = prm->alpha_cut > 0.0 ? prm->alpha_cut : 0.5 * prm->omega * prm->omega;
        P->rec_filter = 1;
    }
    P->omega = prm->omega;
    P->cc.vpar[0] = 4.0 * M_PI / P->vol;
    P->cc.vpar[1] = 1.0 / (4.0 * prm->omega * prm->omega);
    if (prm->gcut > 0.0) {
        P->gcut = prm->gcut;
    } else {
        if (!(prm->eps_g > 0.0 && prm->eps_g < 1.0)) return fail(FTCJ_EINVAL, "eps_g in (0,1) when gcut <= 0");
        P->gcut = 2.0 * prm->omega * std::sqrt(std::log(1.0 / prm->eps_g));
    }
    P->max_dens = prm->max_dens > 0 ? prm->max_dens : 1;
    P->chunk_max = prm->chunk_points > 0 ? prm->chunk_points : kChunkMax;
    if (P->chunk_max < 64 || P->chunk_max > kChunkMax)
        return fail(FTCJ_EINVAL, "chunk_points must be in [64, 4096] (or <= 0 for the default)");
    // basis
    if (basis->ncentre < 1 || !basis->xyz) return fail(FTCJ_EINVAL, "no centres");
    if (basis->nshell < 1 || !basis->shells) return fail(FTCJ_EINVAL, "no shells");
    for (int i = 0; i < 3 * basis->ncentre; ++i)
        if (!finite(basis->xyz[i])) return fail(FTCJ_EINVAL, "non-finite centre");
    P->nshell = basis->nshell;
    P->ncentre = basis->ncentre;
    int ao = 0;
    double amin = 1e300;
    struct Mem {
        int shell, prim;
        ftcj::MemberDev m;
    };
    std::vector<std::vector<Mem>> gmem;
    std::vector<std::pair<int, double>> gkey;
    for (int s = 0; s < basis->nshell; ++s) {
        const ftcj_shell& sh = basis->shells[s];
        if (sh.l < 0) return fail(FTCJ_EINVAL, "negative l");
        if (sh.l > kLmax) return fail(FTCJ_EUNSUPPORTED, "shell l above FTCJ_LMAX");
        if (sh.centre < 0 || sh.centre >= basis->ncentre) return fail(FTCJ_EINVAL, "shell centre out of range");
        if (sh.nprim < 1 || !sh.exps || !sh.coefs) return fail(FTCJ_EINVAL, "shell without primitives");
        int nf = sh.spherical ? 2 * sh.l + 1 : (sh.l + 1) * (sh.l + 2) / 2;
        for (int k = 0; k < sh.nprim; ++k) {
            double al = sh.exps[k];
            if (!(al > 0.0) || !finite(al)) return fail(FTCJ_EINVAL, "exponents must be > 0");
            if (!finite(sh.coefs[k])) return fail(FTCJ_EINVAL, "non-finite coefficient");
            amin = std::min(amin, al);
            int g = -1;
            for (size_t q = 0; q < gkey.size(); ++q)
                if (gkey[q].first == sh.centre && gkey[q].second == al) {
                    g = (int)q;
                    break;
                }
            if (g < 0) {
                g = (int)gkey.size();
                gkey.push_back({sh.centre, al});
                gmem.emplace_back();
            }
            double radial = std::pow(2.0 * al / M_PI, 0.75) * std::pow(4.0 * al, 0.5 * sh.l);
            ftcj::MemberDev m{sh.l, sh.spherical ? 1 : 0, ao, 0, sh.coefs[k] * radial};
            gmem[g].push_back({s, k, m});
        }
        ao += nf;
    }
    P->nao = ao;
    P->ngroup = (int)gkey.size();
    P->groups.clear();
    P->members.clear();
    for (int g = 0; g < P->ngroup; ++g) {
        ftcj::GroupDev gd;
        const double* x = basis->xyz + 3 * gkey[g].first;
        gd.x = x[0];
        gd.y = x[1];
        gd.z = x[2];
        gd.alpha = gkey[g].second;
        gd.centre = gkey[g].first;
        gd.mem0 = (int)P->members.size();
        gd.lmax = 0;
        for (auto& m : gmem[g]) {
            P->members.push_back(m.m);
            P->member_shell.push_back(m.shell);
            P->member_prim.push_back(m.prim);
            P->member_group.push_back(g);
            gd.lmax = std::max(gd.lmax, m.m.l);
        }
        gd.mem1 = (int)P->members.size();
        P->groups.push_back(gd);
    }
    P->nmember = (int)P->members.size();
    // exp(-G^2/4p) must stay representable along the walk
    if (P->gcut * P->gcut / (8.0 * amin) > 600.0)
        return fail(FTCJ_EUNSUPPORTED, "Gcut^2/(4 p_min) above 600: exponents too diffuse for this Gcut");
    int rc = build_walk(P);
    if (rc) return rc;
    if (prm->chunk_points <= 0 && P->precision == FTCJ_PREC_SPLIT && (rc = default_split_chunk(P))) return rc;
    P->n_abs_max = 0;
    for (int v : P->gvec) P->n_abs_max = std::max(P->n_abs_max, std::abs(v));
    if (P->precision == FTCJ_PREC_SPLIT && P->n_abs_max > kSplitNmax)
        return fail(FTCJ_EUNSUPPORTED, "a G index |n_i| above 63: the split form's walks need n^4 exact in FP32 "
                                       "(use FTCJ_PREC_FP64 for this cell and cutoff)");

    FTCJ_CUDA(cudaFree(0));
    int dev = 0;
    FTCJ_CUDA(cudaGetDevice(&dev));
    FTCJ_CUDA(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev));

    if ((rc = upload(P, &P->d_groups, P->groups))) return rc;
    if ((rc = upload(P, &P->d_members, P->members))) return rc;
    if ((rc = upload(P, &P->d_lines, P->lines))) return rc;
    if ((rc = upload(P, &P->d_chunks, P->chunks))) return rc;
    if ((rc = upload(P, &P->d_gvec, P->gvec))) return rc;
    if ((rc = dalloc(P, &P->d_vg, (size_t)P->ng_half))) return rc;
    if ((rc = dalloc(P, &P->d_tw, (size_t)3 * 16 * 16 * 2))) return rc;

    if ((rc = screen_and_sort(P))) return rc;
    if ((rc = keep_record_share(P))) return rc;

    // per-class SoA layout of the Hermite terms
    P->total_terms = 0;
    P->total_terms_g = 0;
    for (int c = 0; c < kNclass; ++c) {
        P->term_base[c] = P->total_terms;
        P->total_terms += (P->class_start[c + 1] - P->class_start[c]) * nterms(c);
        P->term_base_g[c] = P->total_terms_g;
        P->total_terms_g += (P->class_start[c + 1] - P->class_start[c]) * nterms(c + 1);
    }
    P->tiles.clear();
    for (int c = kNclass - 1; c >= 0; --c)
        for (int64_t f = P->class_start[c]; f < P->class_start[c + 1]; f += kTile) {
            int cnt = (int)std::min<int64_t>(kTile, P->class_start[c + 1] - f);
            P->tiles.push_back({c, (int)f, cnt, INFINITY});
        }
    if ((rc = upload(P, &P->d_tiles, P->tiles))) return rc;
    if ((rc = upload_walk_tables(P))) return rc;
    if ((rc = upload_hermite_tables(P))) return rc;
    if ((rc = build_maps(P))) return rc;
    if (prm->pair_gcut_eps > 0.0 && (rc = apply_pair_cutoffs(P))) return rc;
    if (P->precision == FTCJ_PREC_SPLIT && (rc = setup_split(P))) return rc;
    int bps = 1;
    if (P->precision == FTCJ_PREC_SPLIT) {
        if ((rc = rho_walk_split_blocks_per_sm(P, 0, &bps))) return rc;
    } else {
        if ((rc = rho_walk_blocks_per_sm(P, &bps))) return rc;
    }
    int nch = std::max<int>(1, (int)P->chunks.size());
    P->npb = std::max(1, std::min<int>((int)std::max<size_t>(1, P->tiles.size()), P->num_sms * bps / nch));
    if (prm->rho_blocks > 0) {
        P->npb = std::min<int>(prm->rho_blocks, (int)std::max<size_t>(1, P->tiles.size()));
        P->rho_hi_tiles = 0;  // an explicit block count keeps the one-launch walk
    }
    if (P->rho_hi_tiles > 0) {
        // two launches, each filling the GPU with its own persistent blocks
        int bps_hi = 1, bps_lo = 1;
        if ((rc = rho_walk_split_blocks_per_sm(P, 2, &bps_hi))) return rc;
        if ((rc = rho_walk_split_blocks_per_sm(P, 1, &bps_lo))) return rc;
        const int nlo = (int)P->tiles.size() - P->rho_hi_tiles;
        P->npb_hi = std::max(1, std::min(P->rho_hi_tiles, P->num_sms * bps_hi / nch));
        P->npb = P->npb_hi + std::max(1, std::min(nlo, P->num_sms * bps_lo / nch));
    }
    if ((rc = build_rho_schedule(P))) return rc;
    if (P->tc && !P->ortho) return fail(FTCJ_EUNSUPPORTED, "the tensor-core contraction needs an orthorhombic cell");
    if (P->tc && (rc = setup_tc(P))) return rc;
    P->rho_rows = P->tc ? P->tc_ngroups : P->npb;

    size_t nn = (size_t)P->nao * P->nao;
    size_t md = (size_t)P->max_dens;
    if ((rc = dalloc(P, &P->d_D0n, md * P->nk * nn))) return rc;
    if ((rc = dalloc(P, &P->d_J0n, md * P->nk * nn))) return rc;
    if ((rc = dalloc(P, &P->d_cbuf0, 2 * md * P->nk * nn))) return rc;
    if ((rc = dalloc(P, &P->d_cbuf1, 2 * md * P->nk * nn))) return rc;
    // the tensor-core layout pads each class to 16 positions (and the last bulk copy may read 16 past a class)
    if ((rc = dalloc(P, &P->d_Dp, md * (size_t)std::max<long long>(P->total_terms, P->tc_dp_total) + 64))) return rc;
    if ((rc = dalloc(P, &P->d_Jp, md * (size_t)std::max(nch, jp_chunks(P)) * (size_t)P->total_terms))) return rc;
    if ((rc = dalloc(P, &P->d_Jg, md * (size_t)nch * (size_t)P->total_terms_g))) return rc;
    if ((rc = dalloc(P, &P->d_rho_part, 2 * md * (size_t)std::max(P->npb, P->rho_rows) * (size_t)P->ng_half)))
        return rc;
    if ((rc = dalloc(P, &P->d_rho, 2 * md * (size_t)P->ng_half))) return rc;
    if ((rc = dalloc(P, &P->d_W, 2 * md * (size_t)P->ng_half))) return rc;
    P->nEblocks = (int)std::max<int64_t>(1, (P->ng_half + kRedPoints - 1) / kRedPoints);
    if ((rc = dalloc(P, &P->d_Epart, md * (size_t)P->nEblocks))) return rc;
    if ((rc = dalloc(P, &P->d_Dk_stage, 2 * md * P->nk * nn))) return rc;
    if ((rc = dalloc(P, &P->d_Jk_stage, 2 * md * P->nk * nn))) return rc;
    if ((rc = dalloc(P, &P->d_EJ_stage, md))) return rc;
    if ((rc = dalloc(P, &P->d_check, 2))) return rc;
    if ((rc = launch_vg(P))) return rc;
    if ((rc = launch_twiddles(P))) return rc;
    if ((rc = setup_fold(P))) return rc;
    if (prm->classify && (rc = setup_gpw(P))) return rc;
    FTCJ_CUDA(cudaDeviceSynchronize());
    return FTCJ_OK;
}

}  // namespace
}  // namespace ftcj

using namespace ftcj;

extern "C" {

const char* ftcj_strerror(int code) {
    switch (code) {
        case FTCJ_OK: return "ok";
        case FTCJ_EINVAL: return "invalid argument";
        case FTCJ_ENOMEM: return "out of memory";
        case FTCJ_ECUDA: return "CUDA error";
        case FTCJ_ETIMEOUT: return "device wait timed out";
        case FTCJ_EUNSUPPORTED: return "unsupported input";
        default: return "unknown error";
    }
}

const char* ftcj_last_error(void) { return g_last_error.c_str(); }

int ftcj_shard_bounds(const int64_t* class_counts, int precision, int shard_count, int64_t* bounds) {
    if (!class_counts || !bounds || shard_count < 1) return fail(FTCJ_EINVAL, "bad argument");
    for (int c = 0; c < kNclass; ++c)
        if (class_counts[c] < 0) return fail(FTCJ_EINVAL, "negative class count");
    shard_bounds(class_counts, precision, shard_count, bounds);
    return FTCJ_OK;
}

int ftcj_plan_create(const ftcj_cell* cell, const ftcj_basis* basis, const int kmesh[3], const ftcj_params* params,
                     ftcj_plan** out) {
    if (!out) return fail(FTCJ_EINVAL, "null output pointer");
    *out = nullptr;
    ftcj_plan* P = new (std::nothrow) ftcj_plan();
    if (!P) return fail(FTCJ_ENOMEM, "host allocation failed");
    int rc;
    try {
        rc = create(cell, basis, kmesh, params, P);
    } catch (const std::bad_alloc&) {
        rc = fail(FTCJ_ENOMEM, "host allocation failed");
    } catch (...) {
        rc = fail(FTCJ_EINVAL, "unexpected host exception");
    }
    if (rc != FTCJ_OK) {
        free_device(P);
        delete P;
        return rc;
    }
    *out = P;
    return FTCJ_OK;
}

int ftcj_plan_info(const ftcj_plan* P, ftcj_info* o) {
    if (!P || !o) return fail(FTCJ_EINVAL, "null argument");
    std::memset(o, 0, sizeof(*o));
    o->nao = P->nao;
    o->nk = P->nk;
    o->nshell = P->nshell;
    o->ngroup = P->ngroup;
    o->npairs = P->npairs;
    o->npairs_ordered = P->npairs_ordered;
    o->ng_half = P->ng_half;
    o->ng_full = 2 * P->ng_half;
    o->pair_g_units = P->npairs_ordered * o->ng_full;
    for (int c = 0; c < kNclass && c < 5; ++c) o->pairs_by_class[c] = P->class_start[c + 1] - P->class_start[c];
    o->nlines = (int)P->lines.size();
    o->nchunks = (int)P->chunks.size();
    o->gcut = P->gcut;
    o->volume = P->vol;
    o->device_bytes = P->device_bytes;
    o->rho_blocks = P->rho_rows;
    o->n1_table = P->precision == FTCJ_PREC_SPLIT ? split_xtab_entries(P) : 0;
    o->pair_g_units_screened = P->d_rec_gcut ? P->units_screened : o->pair_g_units;
    o->pair_g_units_walked = P->d_rec_gcut ? P->units_walked : o->pair_g_units;
    o->n_abs_max = P->n_abs_max;
    o->grad_split = P->precision == FTCJ_PREC_SPLIT && split_grad_walk_exact(P) ? 1 : 0;
    const bool walks = P->ng_half > 0 && !P->tiles.empty();
    o->rho_walk_launches = walks ? (P->tc ? tc_rho_launches(P, P->max_dens) : (P->rho_hi_tiles > 0 ? 2 : 1)) : 0;
    o->j_walk_launches =
        walks ? (P->tc_j ? tc_j_launches(P, P->max_dens) : (P->precision == FTCJ_PREC_SPLIT ? split_j_launches(P) : 1))
              : 0;
    o->contraction = P->tc ? FTCJ_CONTRACT_TC : FTCJ_CONTRACT_WALK;
    o->tc_mma_flops = P->tc ? P->tc_mma_flops : 0;
    o->j_contraction = P->tc_j ? FTCJ_CONTRACT_TC : FTCJ_CONTRACT_WALK;
    o->tc_j_mma_flops = P->tc_j ? P->tc_j_mma_flops : 0;
    if (P->tc) {
        o->tc_column_axis = P->tc_axis[2];
        o->tc_rows = P->tc_rows;
        o->tc_row_tiles = P->tc_mtiles;
        o->tc_blocks_per_window = P->tc_G;
        o->tc_dens_per_launch = P->tc_nd;
    }
    o->alpha_cut = P->rec_filter ? P->alpha_cut : 0.0;
    if (P->dd) {
        o->dd_pairs = P->dd->npairs;
        o->dd_pairs_ordered = P->dd->npairs_ordered;
        for (int c = 0; c < kNclass && c < 5; ++c)
            o->dd_pairs_by_class[c] = P->dd->class_start[c + 1] - P->dd->class_start[c];
    }
    if (P->gpw) {
        o->gpw_grid[0] = gpw_grid_dim(P, 0);
        o->gpw_grid[1] = gpw_grid_dim(P, 1);
        o->gpw_grid[2] = gpw_grid_dim(P, 2);
        o->gpw_separable = gpw_separable(P);
        o->gpw_launches = gpw_launches(P, P->max_dens);
    }
    return FTCJ_OK;
}

void ftcj_plan_destroy(ftcj_plan* P) {
    if (!P) return;
    release_profiling(P);
    free_device(P);
    delete P;
}

int ftcj_get_gvectors(const ftcj_plan* P, int* n_out) {
    if (!P || !n_out) return fail(FTCJ_EINVAL, "null argument");
    if (!P->gvec.empty()) std::memcpy(n_out, P->gvec.data(), sizeof(int) * P->gvec.size());
    return FTCJ_OK;
}

int ftcj_get_pairs(const ftcj_plan* P, int* out) {
    if (!P || !out) return fail(FTCJ_EINVAL, "null argument");
    if (P->npairs == 0) return FTCJ_OK;
    std::vector<PairDev> h((size_t)P->npairs);
    FTCJ_CUDA(cudaMemcpy(h.data(), P->d_pairs, sizeof(PairDev) * h.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); ++i) {
        out[6 * i + 0] = h[i].ga;
        out[6 * i + 1] = h[i].gb;
        out[6 * i + 2] = h[i].L[0];
        out[6 * i + 3] = h[i].L[1];
        out[6 * i + 4] = h[i].L[2];
        out[6 * i + 5] = h[i].weight;
    }
    return FTCJ_OK;
}

int ftcj_get_groups(const ftcj_plan* P, int* centre, double* exponent, int* members, int* nmember) {
    if (!P) return fail(FTCJ_EINVAL, "null argument");
    if (nmember) *nmember = P->nmember;
    for (int g = 0; g < P->ngroup; ++g) {
        if (centre) centre[g] = P->groups[g].centre;
        if (exponent) exponent[g] = P->groups[g].alpha;
    }
    if (members)
        for (int m = 0; m < P->nmember; ++m) {
            members[3 * m + 0] = P->member_group[m];
            members[3 * m + 1] = P->member_shell[m];
            members[3 * m + 2] = P->member_prim[m];
        }
    return FTCJ_OK;
}

}  // extern "C"
