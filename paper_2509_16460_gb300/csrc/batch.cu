// Batches of independent cells and the walk-shape autotuner.
//
// A batch owns one plan per cell and a small pool of streams.  A build forks
// from the caller's stream with an event, hands the cells to the streams in
// order of decreasing estimated work (pair*G units times densities), each to
// the currently least-loaded stream, and joins every stream back into the
// caller's stream.  Because the fork and join are event edges, the whole
// batch can be captured into one CUDA graph and replayed.
//
// A persistent batch (FTCJ_BATCH_PERSISTENT) runs the per-cell k-mesh
// transforms and Hermite maps on the streams, then the structure-factor
// walks, the potentials and the back-contraction walks of every cell as one
// persistent launch over a shared work queue (walk_split.cu), then the
// per-cell J -> AO maps and transforms on the streams again.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ftcj_internal.h"

namespace {

constexpr int kBatchStreams = 8;

}  // namespace

struct ftcj_batch {
    std::vector<ftcj_plan*> plans;
    ftcj::BatchWalks* walks = nullptr;  // the persistent launch's work queue (persistent batches)
    long long spin = 1LL << 32;         // clock cycles a back-contraction item waits for its cell's potential
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
    if (B->walks) batch_walks_destroy(B->walks);
    B->walks = nullptr;
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

// the cells in order of decreasing work, each on the currently least-loaded stream
std::vector<int> assign(const ftcj_batch* B, const int* ndens, int ns) {
    const int n = (int)B->plans.size();
    std::vector<int> order(n), stream_of(n, 0);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return B->cost[a] * ndens[a] > B->cost[b] * ndens[b]; });
    std::vector<double> load(ns, 0.0);
    for (int c : order) {
        const int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[i] += B->cost[c] * ndens[c];
        stream_of[c] = i;
    }
    return stream_of;
}

int fork(ftcj_batch* B, int ns, cudaStream_t s) {
    FTCJ_CUDA(cudaEventRecord(B->fork, s));
    for (int i = 0; i < ns; ++i) FTCJ_CUDA(cudaStreamWaitEvent(B->streams[i], B->fork, 0));
    return FTCJ_OK;
}

int join(ftcj_batch* B, int ns, cudaStream_t s) {
    for (int i = 0; i < ns; ++i) {
        FTCJ_CUDA(cudaEventRecord(B->join[i], B->streams[i]));
        FTCJ_CUDA(cudaStreamWaitEvent(s, B->join[i], 0));
    }
    return FTCJ_OK;
}

// the persistent form: transforms and maps per cell on the streams, the walks of all cells in one launch
int enqueue_persistent(ftcj_batch* B, const int* ndens, const double* const* Dk, double* const* Jk,
                       double* const* EJ, cudaStream_t s) {
    const int n = (int)B->plans.size();
    for (int c = 0; c < n; ++c)
        if (ndens[c] != B->plans[c]->max_dens)
            return fail(FTCJ_EINVAL, "a persistent batch builds max_dens densities of every cell per call");
    const int ns = std::min(kBatchStreams, std::max(n, 1));
    const std::vector<int> st = assign(B, ndens, ns);
    int rc;
    if ((rc = fork(B, ns, s))) return rc;
    for (int c = 0; c < n; ++c) {
        ftcj_plan* P = B->plans[c];
        if ((rc = launch_fold_build(P, ndens[c], Dk[c], P->d_D0n, B->streams[st[c]]))) return rc;
        if ((rc = launch_hermite_map(P, ndens[c], P->d_D0n, B->streams[st[c]]))) return rc;
    }
    if ((rc = join(B, ns, s))) return rc;
    if ((rc = batch_walks_launch(B->walks, B->plans, B->spin, s))) return rc;
    if ((rc = fork(B, ns, s))) return rc;
    for (int c = 0; c < n; ++c) {
        ftcj_plan* P = B->plans[c];
        cudaStream_t t = B->streams[st[c]];
        if ((rc = launch_jtransform_map(P, ndens[c], P->d_J0n, t))) return rc;
        if ((rc = launch_unfold(P, ndens[c], P->d_J0n, Jk[c], t))) return rc;
        FTCJ_CUDA(cudaMemcpyAsync(EJ[c], P->d_EJ_stage, sizeof(double) * ndens[c], cudaMemcpyDeviceToDevice, t));
    }
    return join(B, ns, s);
}

int enqueue(ftcj_batch* B, const int* ndens, const double* const* Dk, double* const* Jk, double* const* EJ,
            cudaStream_t s) {
    const int n = (int)B->plans.size();
    for (int c = 0; c < n; ++c)
        if (ndens[c] < 1 || !Dk[c] || !Jk[c] || !EJ[c]) return fail(FTCJ_EINVAL, "bad per-cell argument");
    if (B->walks) return enqueue_persistent(B, ndens, Dk, Jk, EJ, s);
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
        if (p.classify) {
            rc = fail(FTCJ_EUNSUPPORTED, "a batch takes long-range plans (classify = 0)");
            break;
        }
        if (flags & FTCJ_BATCH_AUTOTUNE) rc = ftcj_autotune(&cells[c], &bases[c], kmeshes + 3 * c, &params[c], &p,
                                                            nullptr);
        ftcj_plan* P = nullptr;
        if (rc == FTCJ_OK && (flags & FTCJ_BATCH_PERSISTENT) && p.chunk_points <= 0) {
            // one kernel runs every cell's walks: its shared memory (and so its CTAs per SM) follows the
            // longest chunk of the batch, so each cell takes the shortest chunk that holds its G lines
            for (int ch = 512; ch <= 4096; ch *= 2) {
                p.chunk_points = ch;
                rc = ftcj_plan_create(&cells[c], &bases[c], kmeshes + 3 * c, &p, &P);
                if (rc != FTCJ_EUNSUPPORTED) break;
            }
        } else if (rc == FTCJ_OK) {
            rc = ftcj_plan_create(&cells[c], &bases[c], kmeshes + 3 * c, &p, &P);
        }
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
    if (rc == FTCJ_OK && (flags & FTCJ_BATCH_PERSISTENT)) rc = batch_walks_create(B->plans, &B->walks);
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

int ftcj_batch_set_wait(ftcj_batch* B, int wait_log2) {
    if (!B || wait_log2 < 0 || wait_log2 > 40) return fail(FTCJ_EINVAL, "wait_log2 must be 0..40");
    B->spin = 1LL << (wait_log2 ? wait_log2 : 32);
    return FTCJ_OK;
}

int ftcj_batch_status(ftcj_batch* B, int* flags, void* stream) {
    if (!B || !flags) return fail(FTCJ_EINVAL, "null argument");
    *flags = 0;
    if (!B->walks) return FTCJ_OK;
    int rc = batch_walks_error(B->walks, flags, reinterpret_cast<cudaStream_t>(stream));
    if (rc) return rc;
    if (*flags & 1)
        return fail(FTCJ_ETIMEOUT, "a back-contraction item of the persistent batch gave up waiting for its "
                                   "cell's potential");
    return FTCJ_OK;
}

void ftcj_batch_destroy(ftcj_batch* B) {
    if (!B) return;
    release(B);
    delete B;
}

}  // extern "C"
