// Batches of independent cells and the walk-shape autotuner.
//
// A batch owns one plan per cell and a small pool of streams.  A build forks
// from the caller's stream with an event, hands the cells to the streams in
// order of decreasing estimated work (pair*G units times densities), each to
// the currently least-loaded stream, and joins every stream back into the
// caller's stream.  Because the fork and join are event edges, the whole
// batch can be captured into one CUDA graph and replayed.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ftcj_internal.h"

namespace {

constexpr int kBatchStreams = 8;

}  // namespace

struct ftcj_batch {
    std::vector<ftcj_plan*> plans;
    std::vector<double> cost;  // estimated work per density
    cudaStream_t streams[kBatchStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kBatchStreams] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace ftcj;

namespace {

void release(ftcj_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (int i = 0; i < kBatchStreams; ++i) {
        if (B->join[i]) cudaEventDestroy(B->join[i]);
        if (B->streams[i]) cudaStreamDestroy(B->streams[i]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    for (ftcj_plan* p : B->plans) ftcj_plan_destroy(p);
    B->plans.clear();
}

int enqueue(ftcj_batch* B, const int* ndens, const double* const* Dk, double* const* Jk, double* const* EJ,
            cudaStream_t s) {
    const int n = (int)B->plans.size();
    for (int c = 0; c < n; ++c)
        if (ndens[c] < 1 || !Dk[c] || !Jk[c] || !EJ[c]) return fail(FTCJ_EINVAL, "bad per-cell argument");
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return B->cost[a] * ndens[a] > B->cost[b] * ndens[b]; });
    FTCJ_CUDA(cudaEventRecord(B->fork, s));
    const int ns = std::min(kBatchStreams, std::max(n, 1));
    for (int i = 0; i < ns; ++i) FTCJ_CUDA(cudaStreamWaitEvent(B->streams[i], B->fork, 0));
    std::vector<double> load(ns, 0.0);
    for (int c : order) {
        int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[i] += B->cost[c] * ndens[c];
        int rc = ftcj_jbuild(B->plans[c], ndens[c], Dk[c], Jk[c], EJ[c], B->streams[i]);
        if (rc) return rc;
    }
    for (int i = 0; i < ns; ++i) {
        FTCJ_CUDA(cudaEventRecord(B->join[i], B->streams[i]));
        FTCJ_CUDA(cudaStreamWaitEvent(s, B->join[i], 0));
    }
    return FTCJ_OK;
}

}  // namespace

extern "C" {

int ftcj_autotune(const ftcj_cell* cell, const ftcj_basis* basis, const int kmesh[3], const ftcj_params* in,
                  ftcj_params* out, double* best_ms) {
    if (!cell || !basis || !kmesh || !in || !out) return fail(FTCJ_EINVAL, "null argument");
    // 0 = the plan's own default chunk; an explicit chunk equal to it builds
    // the same plan and is skipped
    const int chunks[] = {0, 512, 1024, 2048, 4096};
    int default_chunk = -1;
    ftcj_params best = *in;
    double best_t = 1e300;
    cudaEvent_t e0, e1;
    FTCJ_CUDA(cudaEventCreate(&e0));
    FTCJ_CUDA(cudaEventCreate(&e1));
    int rc = FTCJ_OK;
    bool any = false;
    for (int ch : chunks) {
        if (ch == default_chunk) continue;
        int npb_fill = 0;
        for (int mult = 1; mult <= 2; ++mult) {
            ftcj_params p = *in;
            p.max_dens = 1;
            p.chunk_points = ch;
            p.shard_count = 0;  // a share's walks take the shape of the whole plan's
            p.shard_index = 0;
            // the plan's own count (it fills the GPU, and splits the walk by
            // class where shared memory calls for it), then twice the fill
            p.rho_blocks = mult == 1 ? 0 : 2 * npb_fill;
            ftcj_plan* P = nullptr;
            int r = ftcj_plan_create(cell, basis, kmesh, &p, &P);
            if (r == FTCJ_EUNSUPPORTED) break;  // a G line longer than this chunk
            if (r) {
                rc = r;
                break;
            }
            if (mult == 1) npb_fill = P->npb;
            if (ch == 0) default_chunk = P->chunk_max;
            size_t bytes = sizeof(double) * 2 * (size_t)P->nk * P->nao * P->nao;
            double *Dk = nullptr, *Jk = nullptr, *EJ = nullptr;
            cudaError_t e = cudaMalloc(&Dk, bytes);
            if (e == cudaSuccess) e = cudaMalloc(&Jk, bytes);
            if (e == cudaSuccess) e = cudaMalloc(&EJ, sizeof(double));
            if (e == cudaSuccess) e = cudaMemset(Dk, 0, bytes);
            float t = 1e30f;
            if (e == cudaSuccess) {
                r = ftcj_jbuild(P, 1, Dk, Jk, EJ, nullptr);  // warm-up
                for (int rep = 0; rep < 3 && r == FTCJ_OK; ++rep) {
                    cudaEventRecord(e0, nullptr);
                    r = ftcj_jbuild(P, 1, Dk, Jk, EJ, nullptr);
                    cudaEventRecord(e1, nullptr);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t = std::min(t, ms);
                }
            }
            cudaFree(Dk);
            cudaFree(Jk);
            cudaFree(EJ);
            const int tiles = (int)P->tiles.size();
            ftcj_plan_destroy(P);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune buffers");
                break;
            }
            if (r) {
                rc = r;
                break;
            }
            any = true;
            if (t < best_t) {
                best_t = t;
                best = p;
                best.max_dens = in->max_dens;
                best.shard_count = in->shard_count;
                best.shard_index = in->shard_index;
            }
            if (2 * npb_fill > tiles) break;  // no more blocks than tiles
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (!any) return fail(FTCJ_EUNSUPPORTED, "no walk shape holds the longest G line");
    *out = best;
    if (best_ms) *best_ms = best_t;
    return FTCJ_OK;
}

int ftcj_batch_create(int ncell, const ftcj_cell* cells, const ftcj_basis* bases, const int* kmeshes,
                      const ftcj_params* params, int flags, ftcj_batch** out) {
    if (!out || ncell < 1 || !cells || !bases || !kmeshes || !params) return fail(FTCJ_EINVAL, "bad argument");
    *out = nullptr;
    ftcj_batch* B = new (std::nothrow) ftcj_batch();
    if (!B) return fail(FTCJ_ENOMEM, "host allocation failed");
    int rc = FTCJ_OK;
    for (int c = 0; c < ncell && rc == FTCJ_OK; ++c) {
        ftcj_params p = params[c];
        if (p.shard_count > 1) {
            rc = fail(FTCJ_EINVAL, "a batch takes whole plans (shard_count <= 1)");
            break;
        }
        if (flags & FTCJ_BATCH_AUTOTUNE) rc = ftcj_autotune(&cells[c], &bases[c], kmeshes + 3 * c, &params[c], &p,
                                                            nullptr);
        ftcj_plan* P = nullptr;
        if (rc == FTCJ_OK) rc = ftcj_plan_create(&cells[c], &bases[c], kmeshes + 3 * c, &p, &P);
        if (rc == FTCJ_OK) {
            B->plans.push_back(P);
            B->cost.push_back((double)P->npairs_ordered * (double)(2 * P->ng_half) +
                              4.0 * (double)P->nk * P->nao * P->nao);
        }
    }
    if (rc == FTCJ_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
        for (int i = 0; i < kBatchStreams && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&B->streams[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "batch streams");
    }
    if (rc) {
        release(B);
        delete B;
        return rc;
    }
    *out = B;
    return FTCJ_OK;
}

int ftcj_batch_info(const ftcj_batch* B, int cell, ftcj_info* o) {
    if (!B || cell < 0 || cell >= (int)B->plans.size()) return fail(FTCJ_EINVAL, "bad cell index");
    return ftcj_plan_info(B->plans[cell], o);
}

int ftcj_batch_jbuild(ftcj_batch* B, const int* ndens, const double* const* Dk, double* const* Jk,
                      double* const* EJ, void* stream) {
    if (!B || !ndens || !Dk || !Jk || !EJ) return fail(FTCJ_EINVAL, "null argument");
    return enqueue(B, ndens, Dk, Jk, EJ, reinterpret_cast<cudaStream_t>(stream));
}

int ftcj_batch_capture(ftcj_batch* B, const int* ndens, const double* const* Dk, double* const* Jk,
                       double* const* EJ, void* stream) {
    if (!B || !ndens || !Dk || !Jk || !EJ) return fail(FTCJ_EINVAL, "null argument");
    if (!stream) return fail(FTCJ_EINVAL, "capture needs a stream other than the legacy default stream");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (ftcj_plan* P : B->plans)
        if (P->prof_max > 0) return fail(FTCJ_EINVAL, "disable profiling on the batch's plans before capture");
    FTCJ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(B, ndens, Dk, Jk, EJ, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->graph = g;
    B->exec = x;
    return FTCJ_OK;
}

int ftcj_batch_replay(ftcj_batch* B, void* stream) {
    if (!B) return fail(FTCJ_EINVAL, "null batch");
    if (!B->exec) return fail(FTCJ_EINVAL, "nothing captured");
    FTCJ_CUDA(cudaGraphLaunch(B->exec, reinterpret_cast<cudaStream_t>(stream)));
    return FTCJ_OK;
}

void ftcj_batch_destroy(ftcj_batch* B) {
    if (!B) return;
    release(B);
    delete B;
}

}  // extern "C"
