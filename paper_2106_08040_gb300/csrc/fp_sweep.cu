// Uneven batched sweeps: many instances of different truncation degree and
// stiffness in one submission.
//
// Planning (host): instances are grouped into buckets of equal launch degree
// (L rounded up to a multiple of the bucket width), buckets run largest L
// first, and inside a bucket instances are queued most expensive first
// (longest-processing-time order; cost grows with the anisotropy barrier
// sigma and the field energy b_T |B|max, which set the stiffness).  Each
// bucket is one persistent launch whose CTAs pull instances from a work
// counter, so CTAs that finish early take the next instance.
//
// Running: the bucket launches are forked onto side streams (so a smaller
// bucket fills the SMs a larger one leaves idle at its tail), joined, and
// captured into a CUDA graph that later runs with the same buffers replay.
//
// Autotuning: per bucket, a strided sample of its instances is solved with
// each candidate (Radau stages, refactorisation interval); the fastest
// candidate whose sample converged is kept for that bucket.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>
#include "fp_internal.h"

struct FpBucket {
    int L;            // launch degree
    int start;        // first slot in the order array
    int count;
    int stages;
    int refactor_every;
    float tuned_ms;   // autotune time of the chosen candidate (0 if not tuned)
    unsigned char* d_fac;   // factor scratch of this bucket (five stages or degrees above FP_L_SMEM), else NULL
};

struct fp_sweep {
    fp_ctx* ctx;
    int n;
    std::vector<FpBucket> b;
    std::vector<int> h_order;
    int* d_order = nullptr;       // [n]
    int* d_tune = nullptr;        // [n] sample slots for autotuning
    int* d_queue = nullptr;       // [buckets] work counters
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

void drop_graph(fp_sweep* sw) {
    if (sw->exec) cudaGraphExecDestroy(sw->exec);
    sw->exec = nullptr;
    for (auto& k : sw->key) k = nullptr;
}

int launch_bucket(fp_sweep* sw, int bi, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status,
                  int* d_stats, const int* order, int count, int* queue, cudaStream_t st) {
    fp_ctx* c = sw->ctx;
    const FpBucket& bk = sw->b[bi];
    fp_tol tol = c->tol;
    tol.stages = bk.stages;
    tol.refactor_every = bk.refactor_every;
    DevTab tab{c->d_coef, c->d_src, c->d_lam, c->d_wdiag, c->d_colT, c->d_coef4, c->host.N};
    const size_t sm = fp_solver_smem_bytes(bk.stages, bk.L);
    int max_sm = 0;
    cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if ((int)sm > max_sm) return fp_fail(FP_EUNSUPPORTED, "fp_sweep: %zu bytes of shared memory at L=%d", sm, bk.L);
    int rc = fp_launch_solve(bk.stages, &tab, &c->blk, &c->mat, &c->drv, &tol, d_inst, count, bk.L, d_m, d_dmdt,
                             d_status, d_stats, c->num_sms, st, order, queue, bk.d_fac);
    if (rc != FP_OK) return fp_fail(rc, "fp_sweep: launch at L=%d failed: %s", bk.L, cudaGetErrorString(cudaGetLastError()));
    return FP_OK;
}

// all buckets: memset of the counters, fork, one launch per bucket, join
int enqueue_all(fp_sweep* sw, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status, int* d_stats,
                cudaStream_t st) {
    const int nb = (int)sw->b.size();
    if (cudaMemsetAsync(sw->d_queue, 0, sizeof(int) * nb, st) != cudaSuccess)
        return fp_fail(FP_ECUDA, "fp_sweep_run: counter reset");
    if (cudaEventRecord(sw->fork, st) != cudaSuccess) return fp_fail(FP_ECUDA, "fp_sweep_run: fork");
    for (int i = 1; i < nb; ++i)
        if (cudaStreamWaitEvent(sw->side[i], sw->fork, 0) != cudaSuccess) return fp_fail(FP_ECUDA, "fp_sweep_run: fork wait");
    for (int i = 0; i < nb; ++i) {
        cudaStream_t s = i == 0 ? st : sw->side[i];
        int rc = launch_bucket(sw, i, d_inst, d_m, d_dmdt, d_status, d_stats, sw->d_order + sw->b[i].start,
                               sw->b[i].count, sw->d_queue + i, s);
        if (rc != FP_OK) return rc;
    }
    for (int i = 1; i < nb; ++i) {
        if (cudaEventRecord(sw->join[i], sw->side[i]) != cudaSuccess ||
            cudaStreamWaitEvent(st, sw->join[i], 0) != cudaSuccess)
            return fp_fail(FP_ECUDA, "fp_sweep_run: join");
    }
    return FP_OK;
}

}  // namespace

extern "C" int fp_truncation_degree(const fp_material* mat, const fp_drive* drv, const fp_instance* h_inst, int n,
                                    int L_min, int L_max, int* h_L) {
    if (!mat || !drv || (n > 0 && (!h_inst || !h_L)) || n < 0 || L_min < 2 || L_max < L_min)
        return fp_fail(FP_EINVAL, "fp_truncation_degree: bad argument");
    const double kT = FP_KB * mat->T_B;
    const double amp = std::sqrt(drv->amp[0] * drv->amp[0] + drv->amp[1] * drv->amp[1] + drv->amp[2] * drv->amp[2]);
    for (int i = 0; i < n; ++i) {
        const fp_instance& in = h_inst[i];
        const double V = 3.14159265358979323846 * in.d * in.d * in.d / 6.0;
        const double hb = std::sqrt(in.h_off[0] * in.h_off[0] + in.h_off[1] * in.h_off[1] + in.h_off[2] * in.h_off[2]);
        const double x = in.K * V / kT + V * mat->Ms / kT * (hb + amp);
        double Lr = std::ceil(2.0 + 5.5 * std::sqrt(x > 0.0 ? x : 0.0));
        if (!(Lr >= L_min)) Lr = L_min;          // also for a NaN
        if (Lr > L_max) Lr = L_max;
        h_L[i] = (int)Lr;
    }
    return FP_OK;
}

extern "C" {

int fp_sweep_order(const fp_material* mat, const fp_drive* drv, int L_max, const fp_instance* h_inst, int n,
                   int bucket_width, int* h_order, int* h_bucket_L, int* h_bucket_count, int* n_buckets) {
    if (!mat || !drv || !h_inst || !h_order || !n_buckets) return fp_fail(FP_EINVAL, "fp_sweep_order: NULL argument");
    if (n < 1) return fp_fail(FP_EINVAL, "fp_sweep_order: n=%d", n);
    if (bucket_width < 1) return fp_fail(FP_EINVAL, "fp_sweep_order: bucket_width=%d", bucket_width);
    if (L_max < 2 || L_max > FP_L_MAX_ANY) return fp_fail(FP_EINVAL, "fp_sweep_order: L_max=%d", L_max);
    const double kT = 1.380649e-23 * mat->T_B;
    const double amp = std::sqrt(drv->amp[0] * drv->amp[0] + drv->amp[1] * drv->amp[1] + drv->amp[2] * drv->amp[2]);
    std::vector<int> Lb(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        const fp_instance& in = h_inst[i];
        if (in.L < 2 || in.L > L_max)
            return fp_fail(FP_EINVAL, "fp_sweep_order: instance %d has L=%d outside [2, %d]", i, in.L, L_max);
        Lb[i] = std::min(L_max, (in.L + bucket_width - 1) / bucket_width * bucket_width);
        const double V = 3.14159265358979323846 * in.d * in.d * in.d / 6.0;
        const double sigma = in.K * V / kT, bT = V * mat->Ms / kT;
        const double hb = std::sqrt(in.h_off[0] * in.h_off[0] + in.h_off[1] * in.h_off[1] + in.h_off[2] * in.h_off[2]);
        cost[i] = std::isfinite(sigma + bT * (hb + amp)) ? sigma + bT * (hb + amp) : 0.0;
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (Lb[a] != Lb[b]) return Lb[a] > Lb[b];
        return cost[a] > cost[b];
    });
    int nb = 0;
    for (int s = 0; s < n;) {
        int e = s;
        while (e < n && Lb[idx[e]] == Lb[idx[s]]) ++e;
        if (h_bucket_L) h_bucket_L[nb] = Lb[idx[s]];
        if (h_bucket_count) h_bucket_count[nb] = e - s;
        ++nb;
        s = e;
    }
    std::copy(idx.begin(), idx.end(), h_order);
    *n_buckets = nb;
    return FP_OK;
}

int fp_sweep_plan(fp_ctx* ctx, const fp_instance* h_inst, int n, int bucket_width, fp_sweep** out) {
    if (!ctx || !h_inst || !out) return fp_fail(FP_EINVAL, "fp_sweep_plan: NULL argument");
    *out = nullptr;
    if (n < 1) return fp_fail(FP_EINVAL, "fp_sweep_plan: n=%d", n);
    std::vector<int> idx(n);
    int bL[FP_L_MAX_ANY], bc[FP_L_MAX_ANY], nbk = 0;
    int rc0 = fp_sweep_order(&ctx->mat, &ctx->drv, ctx->L_max, h_inst, n, bucket_width, idx.data(), bL, bc, &nbk);
    if (rc0 != FP_OK) return rc0;
    fp_sweep* sw = new (std::nothrow) fp_sweep();
    if (!sw) return fp_fail(FP_ENOMEM, "fp_sweep_plan: host allocation");
    sw->ctx = ctx;
    sw->n = n;
    sw->h_order = idx;
    for (int k = 0, s = 0; k < nbk; s += bc[k], ++k)
        sw->b.push_back(FpBucket{bL[k], s, bc[k], bL[k] > FP_L_SMEM ? 3 : ctx->tol.stages, ctx->tol.refactor_every,
                                 0.f, nullptr});
    const int nb = (int)sw->b.size();
    int rc = FP_OK;
    // five-stage buckets and buckets above FP_L_SMEM keep their factors in global
    // memory: one scratch per bucket (buckets run concurrently on side streams),
    // one slot per CTA, sized for either stage count the autotuner may pick
    for (auto& bk : sw->b) {
        size_t fb = fp_solver_fac_scratch_bytes(3, bk.L, ctx->num_sms);
        if (bk.L <= FP_L_SMEM) {
            const size_t f5 = fp_solver_fac_scratch_bytes(5, bk.L, ctx->num_sms);
            fb = f5 > fb ? f5 : fb;
        }
        if (rc == FP_OK && fb && cudaMalloc((void**)&bk.d_fac, fb) != cudaSuccess)
            rc = fp_fail(FP_ENOMEM, "fp_sweep_plan: factor scratch at L=%d", bk.L);
    }
    if (cudaMalloc(&sw->d_order, sizeof(int) * n) != cudaSuccess || cudaMalloc(&sw->d_tune, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&sw->d_queue, sizeof(int) * nb) != cudaSuccess)
        rc = fp_fail(FP_ENOMEM, "fp_sweep_plan: cudaMalloc");
    if (rc == FP_OK && cudaMemcpy(sw->d_order, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fp_fail(FP_ECUDA, "fp_sweep_plan: upload");
    sw->side.assign(nb, nullptr);
    sw->join.assign(nb, nullptr);
    if (rc == FP_OK && cudaEventCreateWithFlags(&sw->fork, cudaEventDisableTiming) != cudaSuccess)
        rc = fp_fail(FP_ECUDA, "fp_sweep_plan: event");
    for (int i = 1; i < nb && rc == FP_OK; ++i)
        if (cudaStreamCreateWithFlags(&sw->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sw->join[i], cudaEventDisableTiming) != cudaSuccess)
            rc = fp_fail(FP_ECUDA, "fp_sweep_plan: streams");
    if (rc != FP_OK) {
        fp_sweep_destroy(sw);
        return rc;
    }
    *out = sw;
    return FP_OK;
}

int fp_sweep_destroy(fp_sweep* sw) {
    if (!sw) return FP_OK;
    drop_graph(sw);
    cudaFree(sw->d_order);
    cudaFree(sw->d_tune);
    cudaFree(sw->d_queue);
    for (auto& bk : sw->b) cudaFree(bk.d_fac);
    for (auto s : sw->side)
        if (s) cudaStreamDestroy(s);
    for (auto e : sw->join)
        if (e) cudaEventDestroy(e);
    if (sw->fork) cudaEventDestroy(sw->fork);
    delete sw;
    return FP_OK;
}

int fp_sweep_info(const fp_sweep* sw, int* n_buckets, int* h_L, int* h_count, int* h_stages, int* h_refactor,
                  float* h_tuned_ms) {
    if (!sw || !n_buckets) return fp_fail(FP_EINVAL, "fp_sweep_info: NULL argument");
    *n_buckets = (int)sw->b.size();
    for (size_t i = 0; i < sw->b.size(); ++i) {
        if (h_L) h_L[i] = sw->b[i].L;
        if (h_count) h_count[i] = sw->b[i].count;
        if (h_stages) h_stages[i] = sw->b[i].stages;
        if (h_refactor) h_refactor[i] = sw->b[i].refactor_every;
        if (h_tuned_ms) h_tuned_ms[i] = sw->b[i].tuned_ms;
    }
    return FP_OK;
}

int fp_sweep_run(fp_sweep* sw, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status, int* d_stats,
                 void* stream) {
    if (!sw || !d_inst || !d_status) return fp_fail(FP_EINVAL, "fp_sweep_run: NULL argument");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != sw->ctx->device)
        return fp_fail(FP_EINVAL, "fp_sweep_run: current device is not the context's");
    cudaStream_t st = (cudaStream_t)stream;
    const void* key[6] = {d_inst, d_m, d_dmdt, d_status, d_stats, stream};
    if (!sw->exec || std::memcmp(key, sw->key, sizeof(key)) != 0) {
        drop_graph(sw);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fp_fail(FP_ECUDA, "fp_sweep_run: begin capture (legacy default stream cannot be captured)");
        int rc = enqueue_all(sw, d_inst, d_m, d_dmdt, d_status, d_stats, st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc != FP_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess || !g) return fp_fail(FP_ECUDA, "fp_sweep_run: end capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&sw->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            sw->exec = nullptr;
            return fp_fail(FP_ECUDA, "fp_sweep_run: instantiate: %s", cudaGetErrorString(e));
        }
        std::memcpy(sw->key, key, sizeof(key));
    }
    if (cudaGraphLaunch(sw->exec, st) != cudaSuccess) return fp_fail(FP_ECUDA, "fp_sweep_run: graph launch");
    return FP_OK;
}

int fp_sweep_autotune(fp_sweep* sw, const fp_instance* d_inst, double* d_m, double* d_dmdt, int* d_status,
                      int sample, void* stream) {
    if (!sw || !d_inst || !d_status || sample < 1) return fp_fail(FP_EINVAL, "fp_sweep_autotune: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    static const int cand[4][2] = {{3, 8}, {3, 16}, {5, 8}, {5, 16}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fp_fail(FP_ECUDA, "fp_sweep_autotune: events");
    int rc = FP_OK;
    std::vector<int> stat(sw->n);
    for (size_t bi = 0; bi < sw->b.size() && rc == FP_OK; ++bi) {
        FpBucket& bk = sw->b[bi];
        // strided sample across the bucket's cost order
        const int m = std::min(sample, bk.count);
        std::vector<int> pick(m);
        for (int k = 0; k < m; ++k) pick[k] = sw->h_order[bk.start + (int)((long long)k * bk.count / m)];
        if (cudaMemcpyAsync(sw->d_tune, pick.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = fp_fail(FP_ECUDA, "fp_sweep_autotune: upload");
            break;
        }
        const FpBucket keep = bk;
        float best = -1.f;
        int best_c = -1;
        for (int c = 0; c < 4 && rc == FP_OK; ++c) {
            if (bk.L > FP_L_SMEM && cand[c][0] != 3) continue;     // 3 stages only above FP_L_SMEM
            bk.stages = cand[c][0];
            bk.refactor_every = cand[c][1];
            cudaMemsetAsync(sw->d_queue + bi, 0, sizeof(int), st);
            cudaEventRecord(e0, st);
            rc = launch_bucket(sw, (int)bi, d_inst, d_m, d_dmdt, d_status, nullptr, sw->d_tune, m, sw->d_queue + bi, st);
            cudaEventRecord(e1, st);
            if (rc != FP_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                if (rc == FP_OK) rc = fp_fail(FP_ECUDA, "fp_sweep_autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (cudaMemcpy(stat.data(), d_status, sizeof(int) * sw->n, cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = fp_fail(FP_ECUDA, "fp_sweep_autotune: status read");
                break;
            }
            bool ok = true;
            for (int k = 0; k < m; ++k) ok = ok && stat[pick[k]] == FP_STATUS_OK;
            if (ok && (best < 0.f || ms < best)) {
                best = ms;
                best_c = c;
            }
        }
        bk = keep;
        if (best_c >= 0) {
            bk.stages = cand[best_c][0];
            bk.refactor_every = cand[best_c][1];
            bk.tuned_ms = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graph(sw);
    return rc;
}

}  // extern "C"
