// Public build entry points: argument checks and the order of the steps.
#include <algorithm>

#include "ftcj_internal.h"

using namespace ftcj;

namespace {

// The device address of a host buffer the device can dereference (page-locked
// or managed memory), else nullptr (pageable memory goes through staging).
void* device_alias(const void* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();  // clear the non-sticky error of an unknown pointer
        return nullptr;
    }
    if ((a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) && a.devicePointer)
        return a.devicePointer;
    return nullptr;
}


inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int rho_walk(ftcj_plan* P, int nd, cudaStream_t s) {
    if (P->tc) return launch_tc_rho(P, nd, s);
    return P->precision == FTCJ_PREC_SPLIT ? launch_rho_walk_split(P, nd, s) : launch_rho_walk(P, nd, s);
}

int j_walk(ftcj_plan* P, int nd, const double* W, cudaStream_t s) {
    if (P->tc_j) return launch_tc_j(P, nd, W, s);
    return P->precision == FTCJ_PREC_SPLIT ? launch_j_walk_split(P, nd, W, s) : launch_j_walk(P, nd, W, s);
}

// the whole-build calls need every pair record: a shard plan's partial rho
// and J^{0n} must be summed across the shards between the steps
int whole_plan(const ftcj_plan* P) {
    if (P->shard_count > 1)
        return fail(FTCJ_EINVAL, "a shard plan (shard_count > 1) runs the step calls, with the partial rho and "
                                 "J^{0n} summed across the shards between them");
    return FTCJ_OK;
}

// the step calls expose one potential; a classified plan has two (Sec. 2.6)
int single_potential(const ftcj_plan* P) {
    if (P->rec_filter)
        return fail(FTCJ_EUNSUPPORTED, "a classified plan (compact/diffuse) runs ftcj_jbuild or ftcj_jbuild_host only");
    return FTCJ_OK;
}

int check(const ftcj_plan* P, int ndens, bool batch_limit) {
    if (!P) return fail(FTCJ_EINVAL, "null plan");
    if (ndens < 1) return fail(FTCJ_EINVAL, "ndens must be >= 1");
    if (batch_limit && ndens > P->max_dens) return fail(FTCJ_EINVAL, "ndens above the plan's max_dens");
    return FTCJ_OK;
}

// one batch of <= max_dens densities; every pointer is device memory
int build_batch(ftcj_plan* P, int nd, const double* Dk, double* Jk, double* EJ, cudaStream_t s) {
    int rc;
    cudaEvent_t* ev = nullptr;
    if (P->prof_used < P->prof_max) {
        ev = P->prof_events.data() + (size_t)P->prof_used * kProfEvents;
        ++P->prof_used;
        P->prof_launches += launches_per_batch(P);
    }
    auto mark = [&](int i) -> int {
        if (ev) FTCJ_CUDA(cudaEventRecord(ev[i], s));
        return FTCJ_OK;
    };
    if ((rc = mark(0))) return rc;
    if ((rc = launch_fold_build(P, nd, Dk, P->d_D0n, s))) return rc;
    if ((rc = mark(1))) return rc;
    if ((rc = launch_hermite_map(P, nd, P->d_D0n, s))) return rc;
    if (P->gpw && (rc = launch_hermite_map(P->dd, nd, P->d_D0n, s))) return rc;
    if ((rc = mark(2))) return rc;
    if ((rc = rho_walk(P, nd, s))) return rc;
    if ((rc = mark(8))) return rc;
    if ((rc = launch_gpw_rho(P, nd, s))) return rc;  // the DD records on the grid (classified plans)
    if ((rc = mark(9))) return rc;
    if ((rc = mark(3))) return rc;
    if (P->gpw) {
        if ((rc = launch_rho_reduce(P, nd, P->d_rho, nullptr, nullptr, nullptr, s))) return rc;
        if ((rc = launch_gpw_potential(P, nd, EJ, s))) return rc;
    } else {
        if ((rc = launch_rho_reduce(P, nd, P->d_rho, P->d_W, EJ, nullptr, s))) return rc;
    }
    if ((rc = mark(4))) return rc;
    if ((rc = j_walk(P, nd, P->d_W, s))) return rc;
    if ((rc = mark(10))) return rc;
    if ((rc = launch_gpw_j(P, nd, s))) return rc;
    if ((rc = mark(11))) return rc;
    if ((rc = mark(5))) return rc;
    if ((rc = launch_jtransform_map(P, nd, P->d_J0n, s))) return rc;
    if (P->gpw && (rc = launch_jtransform_map(P->dd, nd, P->d_J0n, s, false))) return rc;
    if ((rc = mark(6))) return rc;
    if ((rc = launch_unfold(P, nd, P->d_J0n, Jk, s))) return rc;
    if ((rc = mark(7))) return rc;
    return FTCJ_OK;
}

}  // namespace

extern "C" {

int ftcj_fold_density(ftcj_plan* P, int ndens, const double* Dk, double* D0n, void* stream) {
    int rc = check(P, ndens, true);
    if (rc) return rc;
    if (!Dk || !D0n) return fail(FTCJ_EINVAL, "null buffer");
    return launch_fold(P, ndens, Dk, D0n, as_stream(stream));
}

int ftcj_rho(ftcj_plan* P, int ndens, const double* D0n, double* rho, void* stream) {
    int rc = check(P, ndens, true);
    if (rc) return rc;
    if (!D0n || !rho) return fail(FTCJ_EINVAL, "null buffer");
    if ((rc = single_potential(P))) return rc;
    cudaStream_t s = as_stream(stream);
    if ((rc = launch_hermite_map(P, ndens, D0n, s))) return rc;
    if ((rc = rho_walk(P, ndens, s))) return rc;
    return launch_rho_reduce(P, ndens, rho, nullptr, nullptr, nullptr, s);
}

int ftcj_potential(ftcj_plan* P, int ndens, const double* rho, double* W, double* EJ, void* stream) {
    int rc = check(P, ndens, false);
    if (rc) return rc;
    if (!rho || !W || !EJ) return fail(FTCJ_EINVAL, "null buffer");
    if ((rc = single_potential(P))) return rc;
    cudaStream_t s = as_stream(stream);
    // batches keep the energy partials inside the plan's scratch
    for (int b0 = 0; b0 < ndens; b0 += P->max_dens) {
        int nd = std::min(P->max_dens, ndens - b0);
        size_t off = (size_t)b0 * P->ng_half * 2;
        if ((rc = launch_rho_reduce(P, nd, nullptr, W + off, EJ + b0, rho + off, s))) return rc;
    }
    return FTCJ_OK;
}

int ftcj_jback(ftcj_plan* P, int ndens, const double* W, double* J0n, void* stream) {
    int rc = check(P, ndens, true);
    if (rc) return rc;
    if (!W || !J0n) return fail(FTCJ_EINVAL, "null buffer");
    if ((rc = single_potential(P))) return rc;
    cudaStream_t s = as_stream(stream);
    if ((rc = j_walk(P, ndens, W, s))) return rc;
    return launch_jtransform_map(P, ndens, J0n, s);
}

int ftcj_unfold_j(ftcj_plan* P, int ndens, const double* J0n, double* Jk, void* stream) {
    int rc = check(P, ndens, true);
    if (rc) return rc;
    if (!J0n || !Jk) return fail(FTCJ_EINVAL, "null buffer");
    return launch_unfold(P, ndens, J0n, Jk, as_stream(stream));
}

int ftcj_jbuild(ftcj_plan* P, int ndens, const double* Dk, double* Jk, double* EJ, void* stream) {
    int rc = check(P, ndens, false);
    if (rc) return rc;
    if ((rc = whole_plan(P))) return rc;
    if (!Dk || !Jk || !EJ) return fail(FTCJ_EINVAL, "null buffer");
    cudaStream_t s = as_stream(stream);
    size_t per = (size_t)P->nk * P->nao * P->nao * 2;  // doubles per complex density
    for (int b0 = 0; b0 < ndens; b0 += P->max_dens) {
        int nd = std::min(P->max_dens, ndens - b0);
        if ((rc = build_batch(P, nd, Dk + b0 * per, Jk + b0 * per, EJ + b0, s))) return rc;
    }
    return FTCJ_OK;
}

int ftcj_jbuild_host(ftcj_plan* P, int ndens, const double* Dk_host, double* Jk_host, double* EJ_host,
                     void* stream) {
    int rc = check(P, ndens, false);
    if (rc) return rc;
    if ((rc = whole_plan(P))) return rc;
    if (!Dk_host || !Jk_host || !EJ_host) return fail(FTCJ_EINVAL, "null buffer");
    cudaStream_t s = as_stream(stream);
    size_t per = (size_t)P->nk * P->nao * P->nao * 2;
    // Page-locked (or managed) buffers are reached from the device over the
    // host link: the k-mesh transforms read D^k and write J^k there directly,
    // so the transfers run inside those kernels instead of as separate copies.
    const double* Dk_dev = static_cast<const double*>(device_alias(Dk_host));
    double* Jk_dev = static_cast<double*>(device_alias(Jk_host));
    for (int b0 = 0; b0 < ndens; b0 += P->max_dens) {
        int nd = std::min(P->max_dens, ndens - b0);
        const double* din = Dk_dev ? Dk_dev + b0 * per : P->d_Dk_stage;
        double* jout = Jk_dev ? Jk_dev + b0 * per : P->d_Jk_stage;
        if (!Dk_dev)
            FTCJ_CUDA(cudaMemcpyAsync(P->d_Dk_stage, Dk_host + b0 * per, sizeof(double) * nd * per,
                                      cudaMemcpyHostToDevice, s));
        if ((rc = build_batch(P, nd, din, jout, P->d_EJ_stage, s))) return rc;
        if (!Jk_dev)
            FTCJ_CUDA(cudaMemcpyAsync(Jk_host + b0 * per, P->d_Jk_stage, sizeof(double) * nd * per,
                                      cudaMemcpyDeviceToHost, s));
        FTCJ_CUDA(cudaMemcpyAsync(EJ_host + b0, P->d_EJ_stage, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    }
    FTCJ_CUDA(cudaStreamSynchronize(s));
    return FTCJ_OK;
}

int ftcj_grad(ftcj_plan* P, int ndens, const double* Dk, double* EJ, double* grad, void* stream) {
    int rc = check(P, ndens, false);
    if (rc) return rc;
    if ((rc = whole_plan(P))) return rc;
    if (!Dk || !EJ || !grad) return fail(FTCJ_EINVAL, "null buffer");
    if ((rc = single_potential(P))) return rc;
    cudaStream_t s = as_stream(stream);
    size_t per = (size_t)P->nk * P->nao * P->nao * 2;
    for (int b0 = 0; b0 < ndens; b0 += P->max_dens) {
        const int nd = std::min(P->max_dens, ndens - b0);
        if ((rc = launch_fold_build(P, nd, Dk + b0 * per, P->d_D0n, s))) return rc;
        if ((rc = launch_hermite_map(P, nd, P->d_D0n, s))) return rc;
        if ((rc = rho_walk(P, nd, s))) return rc;
        if ((rc = launch_rho_reduce(P, nd, P->d_rho, P->d_W, EJ + b0, nullptr, s))) return rc;
        // the degree-(L+1) sums in the plan's form where FP32 holds their powers of n exactly
        const bool split = P->precision == FTCJ_PREC_SPLIT && split_grad_walk_exact(P);
        if ((rc = split ? launch_j_walk_grad_split(P, nd, P->d_W, s) : launch_j_walk_grad(P, nd, P->d_W, s)))
            return rc;
        if ((rc = launch_grad_assemble(P, nd, P->d_D0n, grad + (size_t)b0 * P->ncentre * 3, s))) return rc;
    }
    return FTCJ_OK;
}

int ftcj_plan_status(ftcj_plan* P, int* flags, void* stream) {
    if (!P || !flags) return fail(FTCJ_EINVAL, "null argument");
    cudaStream_t s = as_stream(stream);
    *flags = 0;
    if (P->d_tc_err) {
        FTCJ_CUDA(cudaMemcpyAsync(flags, P->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FTCJ_CUDA(cudaMemsetAsync(P->d_tc_err, 0, sizeof(int), s));
    }
    FTCJ_CUDA(cudaStreamSynchronize(s));
    return FTCJ_OK;
}

int ftcj_check_density(ftcj_plan* P, int ndens, const double* Dk, double* max_imag, double* max_asym,
                       void* stream) {
    int rc = check(P, ndens, true);
    if (rc) return rc;
    if (!Dk || !max_imag || !max_asym) return fail(FTCJ_EINVAL, "null buffer");
    cudaStream_t s = as_stream(stream);
    if ((rc = launch_check_density(P, ndens, Dk, P->d_check, s))) return rc;
    double h[2];
    FTCJ_CUDA(cudaMemcpyAsync(h, P->d_check, sizeof(h), cudaMemcpyDeviceToHost, s));
    FTCJ_CUDA(cudaStreamSynchronize(s));
    *max_imag = h[0];
    *max_asym = h[1];
    return FTCJ_OK;
}

}  // extern "C"
