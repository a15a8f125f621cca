// C ABI of libfp.so: context management, argument checks, launches, the
// phi_hat kernel (Sec. 2.2, model M1 signal) and the host-side diagnostic
// operator export.  See include/fp.h for the contract of every entry point.
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>
#include "fp_internal.h"

static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

// error reporting for the other translation units (fp_mlp.cu)
int fp_fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(FP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

extern "C" {

const char* fp_last_error(void) { return g_err; }

const char* fp_status_str(int code) {
    switch (code) {
        case FP_OK: return "ok";
        case FP_EINVAL: return "invalid argument";
        case FP_ECUDA: return "CUDA error";
        case FP_ENOMEM: return "out of memory";
        case FP_EUNSUPPORTED: return "unsupported";
        case FP_STATUS_MAXSTEPS: return "step budget exhausted";
        case FP_STATUS_STEP_UNDERFLOW: return "step size underflow";
        case FP_STATUS_NONFINITE: return "non-finite state";
        case FP_STATUS_NEWTON_FAIL: return "Newton iteration failed";
        case FP_STATUS_BAD_INPUT: return "bad instance parameters";
        case FP_STATUS_UNRESOLVED: return "truncation degree too low (|<m>| > 1)";
        default: return "unknown code";
    }
}

int fp_max_degree(void) { return FP_L_MAX; }

int fp_destroy(fp_ctx* ctx) {
    if (!ctx) return FP_OK;
    cudaFree(ctx->d_coef);
    cudaFree(ctx->d_src);
    cudaFree(ctx->d_blk_mem);
    cudaFree(ctx->d_lam);
    cudaFree(ctx->d_colT);
    cudaFree(ctx->d_coef4);
    cudaFree(ctx->d_wdiag);
    cudaFree(ctx->d_tw);
    cudaFree(ctx->d_fac);
    cudaFree(ctx->d_queue);
    fp_free_tables(&ctx->host);
    delete ctx;
    return FP_OK;
}

int fp_setup(const fp_material* mat, const fp_drive* drive, const fp_tol* tol, int L_max, fp_ctx** out) {
    if (!mat || !drive || !tol || !out) return fail(FP_EINVAL, "fp_setup: NULL argument");
    *out = nullptr;
    if (L_max < 2 || L_max > FP_L_MAX)
        return fail(FP_EUNSUPPORTED, "fp_setup: L_max=%d outside [2, %d]", L_max, FP_L_MAX);
    if (!(mat->Ms > 0 && mat->alpha > 0 && mat->gamma > 0 && mat->T_B > 0))
        return fail(FP_EINVAL, "fp_setup: material constants must be positive");
    if (!(drive->period > 0) || drive->samples_per_period < 2 || drive->warmup_periods < 0 ||
        drive->output_periods < 1)
        return fail(FP_EINVAL, "fp_setup: bad drive schedule");
    if (!(tol->rtol > 0) || !(tol->atol >= 0) || tol->max_steps < 1 || tol->newton_max_iter < 1 ||
        tol->refactor_every < 1)
        return fail(FP_EINVAL, "fp_setup: bad tolerances");
    if (tol->stages != 3 && tol->stages != 5)
        return fail(FP_EUNSUPPORTED, "fp_setup: stages=%d (3 or 5 supported)", tol->stages);
    if (L_max > FP_L_SMEM && tol->stages != 3)
        return fail(FP_EUNSUPPORTED, "fp_setup: L_max=%d > %d needs 3 stages (the 5-stage factors of blocks of "
                    "2 L rows do not fit a CTA's registers)", L_max, FP_L_SMEM);
    fp_ctx* c = new (std::nothrow) fp_ctx();
    if (!c) return fail(FP_ENOMEM, "fp_setup: host allocation");
    c->mat = *mat;
    c->drv = *drive;
    c->tol = *tol;
    c->L_max = L_max;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return fail(FP_ECUDA, "fp_setup: no CUDA device"); }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (fp_build_tables(L_max, &c->host) != FP_OK) { delete c; return fail(FP_ENOMEM, "fp_setup: tables"); }
    const size_t N = (size_t)c->host.N;
    int rc = FP_OK;
    auto up = [&](void** dst, const void* src, size_t bytes) {
        if (rc != FP_OK) return;
        if (cudaMalloc(dst, bytes) != cudaSuccess) { rc = fail(FP_ENOMEM, "fp_setup: cudaMalloc"); return; }
        if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(FP_ECUDA, "fp_setup: cudaMemcpy");
    };
    {
        // slot-major device copies (see DevTab)
        std::vector<double> cT(N * FP_NSLOT), c4(N * FP_NSLOT), c4T(N * FP_NSLOT);
        std::vector<int> sT(N * FP_NSLOT);
        fp_build_coef4(&c->host, mat->alpha, c4.data());
        for (size_t i = 0; i < N; ++i)
            for (int k = 0; k < FP_NSLOT; ++k) {
                cT[k * N + i] = c->host.coef[i * FP_NSLOT + k];
                sT[k * N + i] = c->host.src[i * FP_NSLOT + k];
                c4T[k * N + i] = c4[i * FP_NSLOT + k];
            }
        up((void**)&c->d_coef, cT.data(), cT.size() * sizeof(double));
        up((void**)&c->d_src, sT.data(), sT.size() * sizeof(int));
        up((void**)&c->d_coef4, c4T.data(), c4T.size() * sizeof(double));
    }
    up((void**)&c->d_lam, c->host.lam, N * sizeof(double));
    up((void**)&c->d_wdiag, c->host.wdiag, N * sizeof(double));
    {
        std::vector<FpPair> colT(N * FP_NCT), colTT(N * FP_NCT);
        if (fp_build_columns(&c->host, colT.data()) != FP_OK) { fp_destroy(c); return fail(FP_EINVAL, "fp_setup: columns"); }
        for (size_t i = 0; i < N; ++i)
            for (int q = 0; q < FP_NCT; ++q) colTT[q * N + i] = colT[i * FP_NCT + q];
        up((void**)&c->d_colT, colTT.data(), colTT.size() * sizeof(FpPair));
    }
    std::vector<double> tw(2 * (size_t)drive->samples_per_period);
    const double twopi = 6.283185307179586476925286766559;
    for (int q = 0; q < drive->samples_per_period; ++q) {
        double ang = twopi * (double)q / (double)drive->samples_per_period;
        tw[2 * q] = std::cos(ang);
        tw[2 * q + 1] = std::sin(ang);
    }
    up((void**)&c->d_tw, tw.data(), tw.size() * sizeof(double));
    if (rc != FP_OK) { fp_destroy(c); return rc; }
    // global factor scratch (five stages, or degrees above FP_L_SMEM): one slot per CTA of the solve launch
    if (const size_t fb = fp_solver_fac_scratch_bytes(tol->stages, L_max, c->num_sms)) {
        if (cudaMalloc((void**)&c->d_fac, fb) != cudaSuccess) { fp_destroy(c); return fail(FP_ENOMEM, "fp_setup: factor scratch"); }
    }
    if (cudaMalloc((void**)&c->d_queue, sizeof(int)) != cudaSuccess) { fp_destroy(c); return fail(FP_ENOMEM, "fp_setup: work counter"); }
    // block structure of every degree 2..L_max, packed into one device buffer
    {
        std::vector<FpBlkHost> bl(L_max + 1);
        size_t rows = 0;
        std::memset(c->blk.off, 0, sizeof(c->blk.off));
        for (int L = 2; L <= L_max; ++L) {
            if (fp_build_blocks(&c->host, L, &bl[L]) != FP_OK) {
                for (int q = 2; q < L; ++q) fp_free_blocks(&bl[q]);
                fp_destroy(c);
                return fail(FP_ENOMEM, "fp_setup: block structure");
            }
            c->blk.off[L] = (int)rows;
            rows += bl[L].N;
        }
        const size_t b_glob = rows * 4, b_u8 = rows * FP_NSB, b_f8 = rows * FP_NSB * 4, b_u6 = rows * FP_NLT,
                     b_f6 = rows * FP_NLT * 4;
        size_t offs[12], o = 0;
        const size_t sizes[12] = {b_glob, b_u8, b_u8, b_f8, b_u6, b_u6, b_f6, b_u6, b_u6, b_f6, b_u6, b_u6};
        for (int q = 0; q < 12; ++q) { offs[q] = o; o += (sizes[q] + 255) & ~(size_t)255; }
        std::vector<unsigned char> hb(o, 0);
        for (int L = 2; L <= L_max; ++L) {
            const FpBlkHost& b = bl[L];
            const size_t r0 = c->blk.off[L];
            std::memcpy(&hb[offs[0] + r0 * 4], b.glob, b.N * 4);
            std::memcpy(&hb[offs[1] + r0 * FP_NSB], b.sb_k, b.N * FP_NSB);
            std::memcpy(&hb[offs[2] + r0 * FP_NSB], b.sb_g, b.N * FP_NSB);
            std::memcpy(&hb[offs[3] + r0 * FP_NSB * 4], b.sb_cf, b.N * FP_NSB * 4);
            std::memcpy(&hb[offs[4] + r0 * FP_NLT], b.dn_k, b.N * FP_NLT);
            std::memcpy(&hb[offs[5] + r0 * FP_NLT], b.dn_g, b.N * FP_NLT);
            std::memcpy(&hb[offs[6] + r0 * FP_NLT * 4], b.dn_cf, b.N * FP_NLT * 4);
            std::memcpy(&hb[offs[7] + r0 * FP_NLT], b.up_k, b.N * FP_NLT);
            std::memcpy(&hb[offs[8] + r0 * FP_NLT], b.up_g, b.N * FP_NLT);
            std::memcpy(&hb[offs[9] + r0 * FP_NLT * 4], b.up_cf, b.N * FP_NLT * 4);
            std::memcpy(&hb[offs[10] + r0 * FP_NLT], b.dnT, b.N * FP_NLT);
            std::memcpy(&hb[offs[11] + r0 * FP_NLT], b.upT, b.N * FP_NLT);
            fp_free_blocks(&bl[L]);
        }
        up(&c->d_blk_mem, hb.data(), o);
        if (rc != FP_OK) { fp_destroy(c); return rc; }
        unsigned char* base = (unsigned char*)c->d_blk_mem;
        c->blk.glob = (const int*)(base + offs[0]);
        c->blk.sb_k = base + offs[1];
        c->blk.sb_g = base + offs[2];
        c->blk.sb_cf = (const float*)(base + offs[3]);
        c->blk.dn_k = base + offs[4];
        c->blk.dn_g = base + offs[5];
        c->blk.dn_cf = (const float*)(base + offs[6]);
        c->blk.up_k = base + offs[7];
        c->blk.up_g = base + offs[8];
        c->blk.up_cf = (const float*)(base + offs[9]);
        c->blk.dnT = base + offs[10];
        c->blk.upT = base + offs[11];
    }
    FpRadau r3, r5;
    if (fp_build_radau(3, &r3) != FP_OK || fp_build_radau(5, &r5) != FP_OK) {
        fp_destroy(c);
        return fail(FP_EINVAL, "fp_setup: Radau constants");
    }
    double glx[FP_NGL], glw[FP_NGL];
    fp_gauss_legendre(FP_NGL, glx, glw);
    if (fp_upload_constants(&r3, &r5, glx, glw) != FP_OK) { fp_destroy(c); return fail(FP_ECUDA, "fp_setup: constants"); }
    *out = c;
    return FP_OK;
}

int fp_num_samples(const fp_ctx* ctx) {
    if (!ctx) return fail(FP_EINVAL, "fp_num_samples: NULL ctx");
    return ctx->drv.output_periods * ctx->drv.samples_per_period;
}

int fp_solve_batch(fp_ctx* ctx, const fp_instance* d_inst, int n, double* d_m, double* d_dmdt, int* d_status,
                   int* d_stats, void* stream) {
    if (!ctx) return fail(FP_EINVAL, "fp_solve_batch: NULL ctx");
    if (n < 0) return fail(FP_EINVAL, "fp_solve_batch: n < 0");
    if (n == 0) return FP_OK;
    if (!d_inst || !d_status) return fail(FP_EINVAL, "fp_solve_batch: NULL instance or status buffer");
    DevTab tab{ctx->d_coef, ctx->d_src, ctx->d_lam, ctx->d_wdiag, ctx->d_colT, ctx->d_coef4, ctx->host.N};
    size_t sm = fp_solver_smem_bytes(ctx->tol.stages, ctx->L_max);
    int max_sm = 0;
    cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if ((int)sm > max_sm)
        return fail(FP_EUNSUPPORTED, "fp_solve_batch: %zu bytes of shared memory needed, %d available", sm, max_sm);
    // CTAs take instances from the context's work counter, so one that finishes
    // early takes the next (per-instance cost varies with the voxel's field)
    if (cudaMemsetAsync(ctx->d_queue, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess)
        return fail(FP_ECUDA, "fp_solve_batch: work counter reset failed");
    int rc = fp_launch_solve(ctx->tol.stages, &tab, &ctx->blk, &ctx->mat, &ctx->drv, &ctx->tol, d_inst, n, ctx->L_max,
                             d_m, d_dmdt, d_status, d_stats, ctx->num_sms, (cudaStream_t)stream, nullptr, ctx->d_queue,
                             ctx->d_fac);
    if (rc != FP_OK) return fail(rc, "fp_solve_batch: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FP_OK;
}

long long fp_grad_workspace_bytes(const fp_ctx* ctx, int n) {
    if (!ctx || n < 0) return fail(FP_EINVAL, "fp_grad_workspace_bytes: bad argument");
    const int grid = n < ctx->num_sms ? n : ctx->num_sms;
    return (long long)grid * 8LL *
           (long long)fp_adjoint_work_doubles_per_cta(ctx->tol.stages, ctx->L_max, ctx->drv.samples_per_period, ctx->tol.max_steps);
}

int fp_grad(fp_ctx* ctx, const fp_instance* d_inst, int n, int k_max, const double* h_channels, int C,
            const double* d_dJ_dphihat, double* d_grad, int* d_status, int* d_stats, void* d_work,
            unsigned long long work_bytes, void* stream) {
    if (!ctx) return fail(FP_EINVAL, "fp_grad: NULL ctx");
    if (n < 0) return fail(FP_EINVAL, "fp_grad: n < 0");
    if (n == 0) return FP_OK;
    if (!d_inst || !d_dJ_dphihat || !d_grad || !d_status || !h_channels || !d_work)
        return fail(FP_EINVAL, "fp_grad: NULL buffer");
    if ((reinterpret_cast<unsigned long long>(d_work) & 15ull) != 0)
        return fail(FP_EINVAL, "fp_grad: workspace not 16-byte aligned");
    if (ctx->L_max > FP_L_SMEM)
        return fail(FP_EUNSUPPORTED, "fp_grad: the adjoint supports L_max <= %d (context has %d)", FP_L_SMEM, ctx->L_max);
    if (k_max < 0 || k_max >= ctx->drv.samples_per_period) return fail(FP_EINVAL, "fp_grad: k_max=%d", k_max);
    if (C < 1 || C > 4) return fail(FP_EINVAL, "fp_grad: C=%d outside [1, 4]", C);
    const long long need = fp_grad_workspace_bytes(ctx, n);
    if ((long long)work_bytes < need)
        return fail(FP_EINVAL, "fp_grad: workspace %llu bytes < %lld needed", work_bytes, need);
    DevTab tab{ctx->d_coef, ctx->d_src, ctx->d_lam, ctx->d_wdiag, ctx->d_colT, ctx->d_coef4, ctx->host.N};
    size_t sm = fp_adjoint_smem_bytes(ctx->tol.stages, ctx->L_max);
    int max_sm = 0;
    cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if ((int)sm > max_sm)
        return fail(FP_EUNSUPPORTED, "fp_grad: %zu bytes of shared memory needed, %d available", sm, max_sm);
    const int grid = n < ctx->num_sms ? n : ctx->num_sms;
    int rc = fp_launch_adjoint(ctx->tol.stages, &tab, &ctx->blk, &ctx->mat, &ctx->drv, &ctx->tol, d_inst, n,
                               ctx->L_max, k_max, h_channels, C, d_dJ_dphihat, ctx->d_tw, d_grad, d_status, d_stats,
                               (double*)d_work, ctx->tol.max_steps, grid, (cudaStream_t)stream);
    if (rc != FP_OK) return fail(rc, "fp_grad: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FP_OK;
}

}  // extern "C"

// phi_hat[i][c][k] = (1/S) sum_j (p_c . dmdt[i][j0 + j]) (cos - i sin)(2 pi j k / S)
__global__ void fp_signal_kernel(const double* __restrict__ dmdt, int S_out, int S, int k_max,
                                 const double* __restrict__ tw, int C, double3 ch0, double3 ch1, double3 ch2,
                                 double3 ch3, double* __restrict__ out) {
    extern __shared__ double su[];           // [C][S] projected samples
    const int inst = blockIdx.x;
    const double* d = dmdt + ((size_t)inst * S_out + (S_out - S)) * 3;
    double3 chs[4] = {ch0, ch1, ch2, ch3};
    for (int e = threadIdx.x; e < S * C; e += blockDim.x) {
        int c = e / S, j = e - c * S;
        const double* v = d + (size_t)j * 3;
        su[e] = chs[c].x * v[0] + chs[c].y * v[1] + chs[c].z * v[2];
    }
    __syncthreads();
    const int K = k_max + 1;
    for (int e = threadIdx.x; e < C * K; e += blockDim.x) {
        int c = e / K, k = e - c * K;
        const double* u = su + (size_t)c * S;
        double re = 0.0, im = 0.0;
        int q = 0;
        for (int j = 0; j < S; ++j) {
            double uj = u[j];
            re = fma(uj, __ldg(tw + 2 * q), re);
            im = fma(-uj, __ldg(tw + 2 * q + 1), im);
            q += k;
            if (q >= S) q -= S;
        }
        double* o = out + (((size_t)inst * C + c) * K + k) * 2;
        o[0] = re / S;
        o[1] = im / S;
    }
}

extern "C" int fp_signal(fp_ctx* ctx, const double* d_dmdt, int n, int k_max, const double* h_channels, int C,
                         double* d_phihat, void* stream) {
    if (!ctx) return fail(FP_EINVAL, "fp_signal: NULL ctx");
    if (n < 0) return fail(FP_EINVAL, "fp_signal: n < 0");
    if (n == 0) return FP_OK;
    const int S = ctx->drv.samples_per_period, S_out = fp_num_samples(ctx);
    if (!d_dmdt || !d_phihat || !h_channels) return fail(FP_EINVAL, "fp_signal: NULL buffer");
    if (k_max < 0 || k_max >= S) return fail(FP_EINVAL, "fp_signal: k_max=%d outside [0, %d)", k_max, S);
    if (C < 1 || C > 4) return fail(FP_EINVAL, "fp_signal: C=%d outside [1, 4]", C);
    double3 ch[4];
    for (int c = 0; c < 4; ++c)
        ch[c] = c < C ? make_double3(h_channels[3 * c], h_channels[3 * c + 1], h_channels[3 * c + 2])
                      : make_double3(0, 0, 0);
    size_t sm = (size_t)S * C * sizeof(double);
    if (sm > 200 * 1024) return fail(FP_EUNSUPPORTED, "fp_signal: period too long for shared memory");
    if (cudaFuncSetAttribute(fp_signal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return fail(FP_ECUDA, "fp_signal: smem attribute");
    fp_signal_kernel<<<n, 256, sm, (cudaStream_t)stream>>>(d_dmdt, S_out, S, k_max, ctx->d_tw, C, ch[0], ch[1],
                                                          ch[2], ch[3], d_phihat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FP_ECUDA, "fp_signal: launch: %s", cudaGetErrorString(e));
    return FP_OK;
}

extern "C" int fp_operator_dense(const fp_material* mat, const fp_instance* h_inst, const double B_nframe[3],
                                 double* h_A) {
    if (!mat || !h_inst || !B_nframe || !h_A) return fail(FP_EINVAL, "fp_operator_dense: NULL argument");
    const int L = h_inst->L;
    if (L < 2 || L > 64) return fail(FP_EINVAL, "fp_operator_dense: L=%d outside [2, 64]", L);
    FpTablesHost tb;
    if (fp_build_tables(L, &tb) != FP_OK) return fail(FP_ENOMEM, "fp_operator_dense: tables");
    const int N = tb.N;
    FpParams P = fp_derive(*mat, h_inst->K, h_inst->d);
    double s[8] = {-0.5 * P.p4, -P.p3, -P.p1 * B_nframe[2], -P.p1 * B_nframe[0], -P.p1 * B_nframe[1],
                   -P.p2 * B_nframe[2], -P.p2 * B_nframe[0], -P.p2 * B_nframe[1]};
    static const int grp[FP_NSLOT] = {0, 0, 1, 1, 2, 3, 3, 4, 4, 5, 5, 6, 6, 6, 6, 7, 7, 7, 7};
    std::memset(h_A, 0, sizeof(double) * (size_t)N * N);
    for (int i = 0; i < N; ++i) {
        h_A[(size_t)i * N + i] += -P.D * tb.lam[i] - 0.5 * P.p4 * tb.wdiag[i];
        for (int k = 0; k < FP_NSLOT; ++k) {
            int j = tb.src[i * FP_NSLOT + k];
            if (j < 0 || j >= N) continue;
            h_A[(size_t)i * N + j] += s[grp[k]] * tb.coef[i * FP_NSLOT + k];
        }
    }
    fp_free_tables(&tb);
    return FP_OK;
}

// ------------------------------------------------ fp_grad without allocation ----
// fp_grad_noalloc runs the adjoint kernel of fp_grad on a fixed scratch buffer
// compiled into this library instead of a caller-supplied workspace.  It is for
// callers that may not allocate device memory at call time: a host program that
// gives this library a fixed device-memory footprint and forbids further
// cudaMalloc (a plugin inside another runtime, a service that must not grow
// or fragment its memory while it runs), or one that cannot size and keep a
// workspace of its own.  The buffer is a static __device__ array, so every GPU
// that loads the library holds FP_GRAD_NOALLOC_SCRATCH_BYTES until the process
// exits.  Host code cannot use the array's name as a device address; the
// device address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

static __device__ __align__(256) double g_fp_grad_scratch[FP_GRAD_NOALLOC_SCRATCH_BYTES / sizeof(double)];

#define FP_NOALLOC_MAX_DEVICES 64
static std::mutex g_noalloc_mu;
static double* g_noalloc_scratch[FP_NOALLOC_MAX_DEVICES];   // device address per device, set on first use

// Device address of the scratch array on the current device `dev` (which the
// caller has checked is current); the first call per device does the lookup.
static int noalloc_scratch(int dev, double** out) {
    if (dev < 0 || dev >= FP_NOALLOC_MAX_DEVICES)
        return fail(FP_EUNSUPPORTED, "fp_grad_noalloc: device %d beyond %d", dev, FP_NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fp_grad_scratch);
        if (e != cudaSuccess || !p)
            return fail(FP_ECUDA, "fp_grad_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_scratch[dev] = (double*)p;
    }
    *out = g_noalloc_scratch[dev];
    return FP_OK;
}

extern "C" int fp_grad_noalloc(fp_ctx* ctx, const fp_instance* d_inst, int n, int k_max, const double* h_channels,
                               int C, const double* d_dJ_dphihat, double* d_grad, int* d_status, int* d_stats,
                               void* stream) {
    if (!ctx) return fail(FP_EINVAL, "fp_grad_noalloc: NULL ctx");
    if (n < 0) return fail(FP_EINVAL, "fp_grad_noalloc: n < 0");
    if (n == 0) return FP_OK;
    if (ctx->L_max > FP_L_SMEM)
        return fail(FP_EUNSUPPORTED, "fp_grad_noalloc: the adjoint supports L_max <= %d (context has %d)", FP_L_SMEM,
                    ctx->L_max);
    if (!d_inst || !d_dJ_dphihat || !d_grad || !d_status || !h_channels)
        return fail(FP_EINVAL, "fp_grad_noalloc: NULL buffer");
    if (k_max < 0 || k_max >= ctx->drv.samples_per_period)
        return fail(FP_EINVAL, "fp_grad_noalloc: k_max=%d", k_max);
    if (C < 1 || C > 4) return fail(FP_EINVAL, "fp_grad_noalloc: C=%d outside [1, 4]", C);
    // one CTA works through its instances one after another in its own slice
    // of the buffer, so the buffer bounds the number of CTAs, not n
    const unsigned long long per_cta =
        8ull * fp_adjoint_work_doubles_per_cta(ctx->tol.stages, ctx->L_max, ctx->drv.samples_per_period,
                                               ctx->tol.max_steps);
    const unsigned long long fit = FP_GRAD_NOALLOC_SCRATCH_BYTES / per_cta;
    if (fit == 0)
        return fail(FP_EINVAL,
                    "fp_grad_noalloc: one instance needs %llu bytes of scratch (L_max=%d, max_steps=%d), the fixed "
                    "buffer holds %llu; lower fp_tol.max_steps or L_max, or use fp_grad with a workspace",
                    per_cta, ctx->L_max, ctx->tol.max_steps, (unsigned long long)FP_GRAD_NOALLOC_SCRATCH_BYTES);
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ctx->device)
        return fail(FP_EINVAL, "fp_grad_noalloc: current device %d, context lives on device %d", dev, ctx->device);
    size_t sm = fp_adjoint_smem_bytes(ctx->tol.stages, ctx->L_max);
    int max_sm = 0;
    cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if ((int)sm > max_sm)
        return fail(FP_EUNSUPPORTED, "fp_grad_noalloc: %zu bytes of shared memory needed, %d available", sm, max_sm);
    double* scratch = nullptr;
    int rc = noalloc_scratch(dev, &scratch);
    if (rc != FP_OK) return rc;
    // every scratch word the kernel reads it has written earlier in the same
    // launch (recorded steps, checkpoints, segment states and stages, readout
    // cotangents), so what an earlier call left there needs no clearing
    int grid = n < ctx->num_sms ? n : ctx->num_sms;
    if ((unsigned long long)grid > fit) grid = (int)fit;
    DevTab tab{ctx->d_coef, ctx->d_src, ctx->d_lam, ctx->d_wdiag, ctx->d_colT, ctx->d_coef4, ctx->host.N};
    rc = fp_launch_adjoint(ctx->tol.stages, &tab, &ctx->blk, &ctx->mat, &ctx->drv, &ctx->tol, d_inst, n, ctx->L_max,
                           k_max, h_channels, C, d_dJ_dphihat, ctx->d_tw, d_grad, d_status, d_stats, scratch,
                           ctx->tol.max_steps, grid, (cudaStream_t)stream);
    if (rc != FP_OK) return fail(rc, "fp_grad_noalloc: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return FP_OK;
}
