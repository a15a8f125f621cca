// BF16 tensor-core MLP for the harmonic surrogate: D = A B^T on tcgen05 with
// TMEM accumulators, TMA-fed shared-memory pipeline and fused epilogues
// (bias, GELU, output de-normalisation, loss gradient, GELU derivative,
// transposed activation copies for the weight-gradient GEMM).
//
// Every GEMM here is "both operands K-major": A is [M][K] and B is [N][K]
// row-major bf16.  The backward products are brought into that form by the
// epilogues, which also store transposed copies (X^T, G^T) and by keeping W^T
// beside W, so one kernel shape serves forward, dX and dW.
//
// Tile: 128 rows (UMMA M = 128), BN columns (64..256), K blocks of 64 bf16 =
// one 128-byte swizzle row; one persistent CTA per SM walks its tiles through
// an STAGES-deep TMA ring.  Warp 0 lane 0 issues TMA, warp 1 lane 0 issues
// tcgen05.mma into one of two TMEM accumulators (warp 1 owns the allocation),
// and the epilogue warps 2.. drain the other accumulator (warp w reads TMEM
// lanes 32 (w % 4) .. + 31, i.e. those tile rows, and one group of columns).
// Every wait is bounded in time; a wait that gives up sets *err and the CTA
// drains its copies and MMAs and frees TMEM before it returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include "../../include/fp.h"

int fp_fail(int code, const char* fmt, ...);

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int EPI_GROUPS = 2;                 // column groups of the epilogue, 4 warps each
constexpr int NTHREADS = 64 + 128 * EPI_GROUPS;   // TMA warp, MMA warp, epilogue warps
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s bound on any single wait

enum Epi : int {
    EPI_HIDDEN_INFER = 0,   // out = bf16(gelu(acc + b))
    EPI_HIDDEN_TRAIN = 1,   // zf = acc + b (f32), out = bf16(gelu(zf)), outT = out^T
    EPI_OUT_INFER = 2,      // outf = (acc + b) * oscale + oshift (f32, columns < N)
    EPI_OUT_TRAIN = 3,      // g = gscale (acc + b - (y - oshift)/oscale); loss += (.)^2; out, outT = bf16(g)
    EPI_DX_GELU = 4,        // g = acc * gelu'(zin); out, outT = bf16(g)
    EPI_DW = 5,             // outf = acc (f32)
    EPI_OUT_ENSEMBLE = 6,   // y1 = (acc + b) * oscale + oshift; outf holds y0 and receives (y0 + y1) / 2;
                            // rowacc[row] += (|y0 - y1|^2, |mean|^2)
};

struct EpiParams {
    int M, N;                       // valid extent of D
    const float* bias;              // [N]
    __nv_bfloat16* out; int ldo;    // [M][ldo]
    __nv_bfloat16* outT; int ldt;   // [N][ldt]
    float* outf; int ldf;           // [M][ldf]
    const float* zin; int ldz;      // [M][ldz] pre-activation (EPI_DX_GELU)
    const float* y; int ldy;        // [M][ldy] raw targets (EPI_OUT_TRAIN)
    const float* oshift;            // [N]
    const float* oscale;            // [N]
    float* loss;                    // scalar accumulator (EPI_OUT_TRAIN)
    float* rowacc;                  // [M][2] per-row sums (EPI_OUT_ENSEMBLE)
    float gscale;
    int* err;
    int nk;                         // number of 64-wide K blocks
};

// ------------------------------------------------------------- PTX helpers ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false if the phase did not complete within WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (16 B)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);            // start address
    d |= (uint64_t)1 << 16;                              // leading byte offset (16 B >> 4)
    d |= (uint64_t)(1024 >> 4) << 32;                    // stride byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                              // swizzle: 128 B
    return d;
}

// instruction descriptor, kind::f16: A, B bf16, D f32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// erf by Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7, far below the BF16
// resolution of the activations): erf(x) = 1 - t (a1 + t (a2 + ... a5 t)) exp(-x^2),
// t = 1 / (1 + p x) for x >= 0, odd in x
__device__ __forceinline__ float erf_as(float z) {
    const float x = fabsf(z);
    const float t = __frcp_rn(fmaf(0.3275911f, x, 1.f));
    float y = fmaf(1.061405429f, t, -1.453152027f);
    y = fmaf(y, t, 1.421413741f);
    y = fmaf(y, t, -0.284496736f);
    y = fmaf(y, t, 0.254829592f);
    const float e = 1.f - y * t * __expf(-x * x);
    return copysignf(e, z);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erf_as(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erf_as(x * 0.70710678118654752f)) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

template <int BN> struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // one persistent CTA per SM: the ring takes most of the shared memory
    static constexpr int STAGES = (196 * 1024) / STAGE > 8 ? 8 : (196 * 1024) / STAGE;
    static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;   // one accumulator
    static constexpr int SMEM = STAGES * STAGE + 1024 /* align */ + 256 /* barriers */;
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms need 1024-byte tiles");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
};

constexpr int EPI_WARPS = 4 * EPI_GROUPS;    // warps 2 ..
constexpr int MAX_EPI_COLS = 1024;           // bias / output scale staged in shared memory

// ---------------------------------------------------------------- epilogue ----
// sb, ssc, ssh: bias, output scale and shift of this chunk's 16 columns (shared memory)
template <int EPI>
__device__ __forceinline__ void epilogue_chunk(const EpiParams& P, int row, int col0, float* v, const float* sb,
                                               const float* ssc, const float* ssh, float* racc) {
    const bool rv = row < P.M;
    if (EPI == EPI_OUT_ENSEMBLE) {
        if (!rv) return;
        float* o = P.outf + (size_t)row * P.ldf + col0;
        float y0[16];
        const bool full = col0 + 16 <= P.N && ((P.ldf & 3) == 0);
        if (full) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
                const float4 a = *(const float4*)(o + i);
                y0[i] = a.x; y0[i + 1] = a.y; y0[i + 2] = a.z; y0[i + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) y0[i] = col0 + i < P.N ? o[i] : 0.f;
        }
        float mn[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const bool cv = col0 + i < P.N;
            const float y1 = (v[i] + sb[i]) * ssc[i] + ssh[i];
            const float d = cv ? y0[i] - y1 : 0.f;
            mn[i] = cv ? 0.5f * (y0[i] + y1) : 0.f;
            racc[0] = fmaf(d, d, racc[0]);
            racc[1] = fmaf(mn[i], mn[i], racc[1]);
        }
        if (full) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) *(float4*)(o + i) = make_float4(mn[i], mn[i + 1], mn[i + 2], mn[i + 3]);
        } else {
            for (int i = 0; i < 16 && col0 + i < P.N; ++i) o[i] = mn[i];
        }
        return;
    }
    if (EPI == EPI_DW) {
        if (!rv) return;
        float* o = P.outf + (size_t)row * P.ldf + col0;
        if (col0 + 16 <= P.N) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) *(float4*)(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
            for (int i = 0; i < 16 && col0 + i < P.N; ++i) o[i] = v[i];
        }
        return;
    }
    if (EPI == EPI_OUT_INFER) {
        if (!rv) return;
        float* o = P.outf + (size_t)row * P.ldf + col0;
        float r[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) r[i] = (v[i] + sb[i]) * ssc[i] + ssh[i];
        if (col0 + 16 <= P.N && ((P.ldf & 3) == 0)) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) *(float4*)(o + i) = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
        } else {
            for (int i = 0; i < 16 && col0 + i < P.N; ++i) o[i] = r[i];
        }
        return;
    }
    float g[16];
    float lsum = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int c = col0 + i;
        const bool cv = c < P.N;
        float r = 0.f;
        if (EPI == EPI_HIDDEN_INFER || EPI == EPI_HIDDEN_TRAIN) {
            const float z = v[i] + sb[i];
            if (EPI == EPI_HIDDEN_TRAIN && rv && cv) P.outf[(size_t)row * P.ldf + c] = z;
            r = gelu(z);
        } else if (EPI == EPI_OUT_TRAIN) {
            if (rv && cv) {
                const float z = v[i] + sb[i];
                const float t = (__ldg(P.y + (size_t)row * P.ldy + c) - ssh[i]) / ssc[i];
                const float d = z - t;
                lsum += d * d;
                r = P.gscale * d;
            }
        } else if (EPI == EPI_DX_GELU) {
            if (rv && cv) r = v[i] * gelu_grad(__ldg(P.zin + (size_t)row * P.ldz + c));
        }
        g[i] = (rv && cv) ? r : 0.f;
    }
    if (EPI == EPI_OUT_TRAIN) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((threadIdx.x & 31) == 0 && lsum != 0.f) atomicAdd(P.loss, lsum);
    }
    if (rv) {
        __nv_bfloat16* o = P.out + (size_t)row * P.ldo + col0;
        if (col0 + 16 <= P.N) {
            __align__(16) __nv_bfloat16 b[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) b[i] = __float2bfloat16_rn(g[i]);
            *(uint4*)o = *(const uint4*)b;
            *(uint4*)(o + 8) = *(const uint4*)(b + 8);
        } else {
            for (int i = 0; i < 16 && col0 + i < P.N; ++i) o[i] = __float2bfloat16_rn(g[i]);
        }
    }
    if (EPI != EPI_HIDDEN_INFER && P.outT) {
        // transposed copy: for each column, the warp's 32 rows are contiguous
        for (int i = 0; i < 16; ++i) {
            const int c = col0 + i;
            if (c < P.N && rv) P.outT[(size_t)c * P.ldt + row] = __float2bfloat16_rn(g[i]);
        }
    }
}

// ------------------------------------------------------------------ kernel ----
// Persistent: one CTA per SM walks the output tiles (tile t -> row block
// t / ntn, column block t % ntn, so neighbouring tiles share their A rows).
// Warp 0 lane 0 streams K blocks of every tile through the TMA ring, warp 1
// lane 0 issues the MMAs into one of two TMEM accumulators, and the epilogue
// warps drain the other accumulator, so the epilogue of tile u overlaps the
// main loop of tile u + 1.
template <int BN, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
mlp_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, EpiParams P) {
    using C = Cfg<BN>;
    constexpr int ST = C::STAGES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* tiles = smem;
    uint64_t* bars = (uint64_t*)(smem + ST * C::STAGE);   // full[ST], empty[ST], acc_full[2], acc_empty[2], drain
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * ST + 5);
    int* abort_flag = (int*)(tmem_slot + 1);
    __shared__ float s_bias[MAX_EPI_COLS], s_osc[MAX_EPI_COLS], s_osh[MAX_EPI_COLS];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = P.nk;
    const int ntn = (P.N + BN - 1) / BN, ntm = (P.M + BM - 1) / BM, ntiles = ntn * ntm;
    for (int j = threadIdx.x; j < MAX_EPI_COLS; j += NTHREADS) {
        const bool in = j < P.N;
        s_bias[j] = (in && P.bias) ? P.bias[j] : 0.f;
        s_osc[j] = (in && P.oscale) ? P.oscale[j] : 1.f;
        s_osh[j] = (in && P.oshift) ? P.oshift[j] : 0.f;
    }
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + ST);
    const uint32_t accf0 = smem_u32(bars + 2 * ST), acce0 = smem_u32(bars + 2 * ST + 2);
    const uint32_t drain = smem_u32(bars + 2 * ST + 4);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * ST + 2; ++s) mbar_init(smem_u32(bars + s), 1);
        mbar_init(acce0, EPI_WARPS);
        mbar_init(acce0 + 8, EPI_WARPS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)(2 * C::TMEM_COLS))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int* abort_v = abort_flag;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer over all tiles of this CTA
            long long g = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x) {
                const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % ST);
                    if (g >= ST && !mbar_wait(empty0 + 8 * s, (uint32_t)(((g / ST) - 1) & 1))) {
                        atomicOr(P.err, 1);
                        *abort_v = 1;
                    }
                    if (*abort_v) break;
                    const uint32_t sa = smem_u32(tiles + s * C::STAGE);
                    mbar_expect_tx(full0 + 8 * s, C::STAGE);
                    tma_load_2d(sa, &mapA, full0 + 8 * s, kb * BK, m0);
                    tma_load_2d(sa + C::A_BYTES, &mapB, full0 + 8 * s, kb * BK, n0);
                }
            }
            if (*abort_v)   // let the copies still in flight land before the CTA exits
                for (long long h = g - 1; h >= 0 && h >= g - ST; --h)
                    mbar_wait(full0 + 8 * (int)(h % ST), (uint32_t)((h / ST) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            long long g = 0;
            int u = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_v; t += gridDim.x, ++u) {
                const int b = u & 1, q = u >> 1;
                if (q >= 1 && !mbar_wait(acce0 + 8 * b, (uint32_t)((q - 1) & 1))) {
                    atomicOr(P.err, 8);
                    *abort_v = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * C::TMEM_COLS);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % ST);
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)((g / ST) & 1)) || *abort_v) {
                        atomicOr(P.err, 2);
                        *abort_v = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + s * C::STAGE);
                    const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        mma_bf16(acc, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc, (kb | k) != 0);
                    mma_commit(empty0 + 8 * s);        // frees the stage once these MMAs are done
                }
                if (*abort_v) break;
                mma_commit(accf0 + 8 * b);             // accumulator b complete
            }
            mma_commit(drain);                         // every MMA this thread issued has completed
            if (!mbar_wait(drain, 0)) atomicOr(P.err, 16);
        }
    } else {
        // epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 and one column group
        const int lg = warp & 3, grp = (warp - 2) >> 2;
        constexpr int NCH = BN / 16;                   // 16-column chunks of a tile
        const int c_lo = 16 * (grp * NCH / EPI_GROUPS), c_hi = 16 * ((grp + 1) * NCH / EPI_GROUPS);
        int u = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++u) {
            const int b = u & 1, q = u >> 1;
            const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
            const bool ok = !*abort_v && mbar_wait(accf0 + 8 * b, (uint32_t)(q & 1));
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicOr(P.err, 4);
                *abort_v = 1;
                break;
            }
            tc_fence_after();
            const int row = m0 + lg * 32 + lane;
            const uint32_t tw = tmem + (uint32_t)(b * C::TMEM_COLS) + ((uint32_t)(lg * 32) << 16);
            float racc[2] = {0.f, 0.f};
#pragma unroll 1
            for (int c = c_lo; c < c_hi; c += 16) {
                float v[16];
                tmem_ld16(tw + c, v);
                if (n0 + c < P.N)
                    epilogue_chunk<EPI>(P, row, n0 + c, v, s_bias + n0 + c, s_osc + n0 + c, s_osh + n0 + c, racc);
            }
            if (EPI == EPI_OUT_ENSEMBLE && row < P.M) {
                atomicAdd(P.rowacc + 2 * (size_t)row, racc[0]);
                atomicAdd(P.rowacc + 2 * (size_t)row + 1, racc[1]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * b) : "memory");
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)(2 * C::TMEM_COLS))
                     : "memory");
    }
}

// ------------------------------------------------------------ tensor maps ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// row-major bf16 [rows][cols] (cols contiguous, ld elements per row), box = box_rows x 64
int make_map(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return FP_ECUDA;
    if (((uintptr_t)base & 15) || (ld * 2) % 16 || rows < 1 || cols < 1) return FP_EINVAL;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FP_OK : FP_ECUDA;
}

template <int BN, int EPI>
int launch_t(const CUtensorMap& a, const CUtensorMap& b, const EpiParams& P, int M, int N, cudaStream_t st) {
    using C = Cfg<BN>;
    if (cudaFuncSetAttribute(mlp_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
        cudaSuccess)
        return FP_ECUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (long long)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    mlp_gemm_kernel<BN, EPI><<<grid, NTHREADS, C::SMEM, st>>>(a, b, P);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ECUDA;
}

template <int EPI>
int launch_bn(int BN, const CUtensorMap& a, const CUtensorMap& b, const EpiParams& P, int M, int N,
              cudaStream_t st) {
    switch (BN) {
        case 64: return launch_t<64, EPI>(a, b, P, M, N, st);
        case 128: return launch_t<128, EPI>(a, b, P, M, N, st);
        case 160: return launch_t<160, EPI>(a, b, P, M, N, st);
        case 256: return launch_t<256, EPI>(a, b, P, M, N, st);
        default: return FP_EINVAL;
    }
}

// D[M][N] = A[M][K] B[N][K]^T with epilogue `epi`; A, B bf16 row-major with
// leading dimensions lda, ldb (elements); BN is the tile width.
int gemm(int epi, int BN, const void* A, int lda, const void* B, int ldb, int M, int N, int K, const EpiParams& P_in,
         cudaStream_t st) {
    if (M < 1 || N < 1 || K < 1) return FP_EINVAL;
    if (N > MAX_EPI_COLS && (P_in.bias || P_in.oscale || P_in.oshift)) return FP_EINVAL;
    CUtensorMap ma, mb;
    int rc = make_map(&ma, A, M, K, lda, BM);
    if (rc != FP_OK) return rc;
    rc = make_map(&mb, B, N, K, ldb, BN);
    if (rc != FP_OK) return rc;
    EpiParams P = P_in;
    P.M = M;
    P.N = N;
    P.nk = (K + BK - 1) / BK;
    switch (epi) {
        case EPI_HIDDEN_INFER: return launch_bn<EPI_HIDDEN_INFER>(BN, ma, mb, P, M, N, st);
        case EPI_HIDDEN_TRAIN: return launch_bn<EPI_HIDDEN_TRAIN>(BN, ma, mb, P, M, N, st);
        case EPI_OUT_INFER: return launch_bn<EPI_OUT_INFER>(BN, ma, mb, P, M, N, st);
        case EPI_OUT_TRAIN: return launch_bn<EPI_OUT_TRAIN>(BN, ma, mb, P, M, N, st);
        case EPI_DX_GELU: return launch_bn<EPI_DX_GELU>(BN, ma, mb, P, M, N, st);
        case EPI_DW: return launch_bn<EPI_DW>(BN, ma, mb, P, M, N, st);
        case EPI_OUT_ENSEMBLE: return launch_bn<EPI_OUT_ENSEMBLE>(BN, ma, mb, P, M, N, st);
        default: return FP_EINVAL;
    }
}

// ------------------------------------------------------- small kernels ----
// x0[m][j] = bf16((x[m][j] - shift_j) * scale_j), j < 7, zero up to 64; and,
// if x0T is given, x0T[j][m] (rows 0..63, leading dimension ldt)
__global__ void prep_input_kernel(const float* __restrict__ x, int q, const float* __restrict__ shift,
                                  const float* __restrict__ scale, __nv_bfloat16* __restrict__ x0,
                                  __nv_bfloat16* __restrict__ x0T, int ldt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)q * FP_SUR_KIN) return;
    const int m = (int)(e / FP_SUR_KIN), j = (int)(e - (long long)m * FP_SUR_KIN);
    float v = 0.f;
    if (j < FP_SUR_IN) v = (x[(size_t)m * FP_SUR_IN + j] - shift[j]) * scale[j];
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    x0[e] = b;
    if (x0T) x0T[(size_t)j * ldt + m] = b;
}

// db[n] = sum_m gT[n][m]: one warp per row
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ gT, int ldt, int q, int N, float* __restrict__ db) {
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    float s = 0.f;
    for (int m = lane; m < q; m += 32) s += __bfloat162float(gT[(size_t)n * ldt + m]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[n] = s;
}

struct AdamArgs {
    float lr, b1, b2, eps, c1, c2;   // c1 = 1 - b1^t, c2 = 1 - b2^t
    int step;
};

__device__ __forceinline__ float adam_update(float p, float g, float& m, float& v, const AdamArgs& a) {
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    return p - a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
}

// one layer: master W [N][K] (and b [N]) updated in place, bf16 W and W^T refreshed
__global__ void adam_layer_kernel(float* __restrict__ W, const float* __restrict__ gW, float* __restrict__ mW,
                                  float* __restrict__ vW, float* __restrict__ b, const float* __restrict__ gb,
                                  float* __restrict__ mb, float* __restrict__ vb, __nv_bfloat16* __restrict__ Wb,
                                  __nv_bfloat16* __restrict__ WTb, int N, int K, AdamArgs a) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long NK = (long long)N * K;
    if (e < NK) {
        float p = W[e];
        if (a.step > 0) {
            float m = mW[e], v = vW[e];
            p = adam_update(p, gW[e], m, v, a);
            mW[e] = m; vW[e] = v; W[e] = p;
        }
        const int n = (int)(e / K), k = (int)(e - (long long)n * K);
        const __nv_bfloat16 pb = __float2bfloat16_rn(p);
        Wb[e] = pb;
        if (WTb) WTb[(size_t)k * N + n] = pb;
    } else if (e < NK + N && a.step > 0) {
        const int n = (int)(e - NK);
        float m = mb[n], v = vb[n];
        b[n] = adam_update(b[n], gb[n], m, v, a);
        mb[n] = m; vb[n] = v;
    }
}

const int KL[FP_SUR_LAYERS] = {FP_SUR_KIN, FP_SUR_HIDDEN, FP_SUR_HIDDEN, FP_SUR_HIDDEN, FP_SUR_HIDDEN};
const int NL[FP_SUR_LAYERS] = {FP_SUR_HIDDEN, FP_SUR_HIDDEN, FP_SUR_HIDDEN, FP_SUR_HIDDEN, FP_SUR_OUT};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct InferWs {
    __nv_bfloat16 *x0, *h[2];
};

size_t infer_ws(long long q, unsigned char* base, InferWs* w) {
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base ? base + o : nullptr; o += al256(bytes); return p; };
    InferWs t;
    t.x0 = (__nv_bfloat16*)take((size_t)q * FP_SUR_KIN * 2);
    t.h[0] = (__nv_bfloat16*)take((size_t)q * FP_SUR_HIDDEN * 2);
    t.h[1] = (__nv_bfloat16*)take((size_t)q * FP_SUR_HIDDEN * 2);
    if (w) *w = t;
    return o;
}

struct TrainWs {
    __nv_bfloat16 *x0, *x0T;                              // [q][64], [64][ldt]
    float* z[FP_SUR_LAYERS - 1];                          // [q][512] pre-activations
    __nv_bfloat16* h[FP_SUR_LAYERS - 1];                  // [q][512] activations (inputs of layers 1..4)
    __nv_bfloat16* hT[FP_SUR_LAYERS - 1];                 // [512][ldt]
    __nv_bfloat16 *g4, *g4T;                              // [q][800], [800][ldt]
    __nv_bfloat16 *g[2], *gT[2];                          // [q][512], [512][ldt] ping-pong
    int ldt;
};

size_t train_ws(long long q, unsigned char* base, TrainWs* w) {
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base ? base + o : nullptr; o += al256(bytes); return p; };
    TrainWs t;
    t.ldt = (int)((q + 7) / 8 * 8);
    t.x0 = (__nv_bfloat16*)take((size_t)q * FP_SUR_KIN * 2);
    t.x0T = (__nv_bfloat16*)take((size_t)FP_SUR_KIN * t.ldt * 2);
    for (int l = 0; l < FP_SUR_LAYERS - 1; ++l) {
        t.z[l] = (float*)take((size_t)q * FP_SUR_HIDDEN * 4);
        t.h[l] = (__nv_bfloat16*)take((size_t)q * FP_SUR_HIDDEN * 2);
        t.hT[l] = (__nv_bfloat16*)take((size_t)FP_SUR_HIDDEN * t.ldt * 2);
    }
    t.g4 = (__nv_bfloat16*)take((size_t)q * FP_SUR_OUT * 2);
    t.g4T = (__nv_bfloat16*)take((size_t)FP_SUR_OUT * t.ldt * 2);
    for (int i = 0; i < 2; ++i) {
        t.g[i] = (__nv_bfloat16*)take((size_t)q * FP_SUR_HIDDEN * 2);
        t.gT[i] = (__nv_bfloat16*)take((size_t)FP_SUR_HIDDEN * t.ldt * 2);
    }
    if (w) *w = t;
    return o;
}

EpiParams epi0(int* err) {
    EpiParams P;
    std::memset(&P, 0, sizeof(P));
    P.err = err;
    return P;
}

}  // namespace

extern "C" {

long long fp_surrogate_workspace_bytes(int q, int training) {
    if (q < 1) return fp_fail(FP_EINVAL, "fp_surrogate_workspace_bytes: q=%d", q);
    if (training == 2) return (long long)(infer_ws(q, nullptr, nullptr) + al256((size_t)q * 2 * sizeof(float)));
    return (long long)(training ? train_ws(q, nullptr, nullptr) : infer_ws(q, nullptr, nullptr));
}

// one network's forward pass; the last layer's epilogue is EPI_OUT_INFER into
// d_y, or EPI_OUT_ENSEMBLE folding this network's output into the mean in d_y
static int infer_member(const fp_surrogate* net, const float* d_x, int q, float* d_y, const InferWs& w, int* d_err,
                        float* rowacc, cudaStream_t st, const char* who) {
    for (int l = 0; l < FP_SUR_LAYERS; ++l)
        if (!net->W[l] || !net->b[l]) return fp_fail(FP_EINVAL, "%s: layer %d not set", who, l);
    if (!net->in_shift || !net->in_scale || !net->out_shift || !net->out_scale)
        return fp_fail(FP_EINVAL, "%s: normalisation not set", who);
    const long long tot = (long long)q * FP_SUR_KIN;
    prep_input_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d_x, q, net->in_shift, net->in_scale, w.x0,
                                                                       nullptr, 0);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "%s: input kernel launch", who);
    const __nv_bfloat16* x = w.x0;
    for (int l = 0; l < FP_SUR_LAYERS; ++l) {
        EpiParams P = epi0(d_err);
        P.bias = net->b[l];
        int rc;
        if (l < FP_SUR_LAYERS - 1) {
            P.out = w.h[l & 1];
            P.ldo = FP_SUR_HIDDEN;
            rc = gemm(EPI_HIDDEN_INFER, 256, x, KL[l], net->W[l], KL[l], q, NL[l], KL[l], P, st);
            x = w.h[l & 1];
        } else {
            P.outf = d_y;
            P.ldf = FP_SUR_OUT;
            P.oshift = net->out_shift;
            P.oscale = net->out_scale;
            P.rowacc = rowacc;
            rc = gemm(rowacc ? EPI_OUT_ENSEMBLE : EPI_OUT_INFER, 160, x, KL[l], net->W[l], KL[l], q, NL[l], KL[l], P,
                      st);
        }
        if (rc != FP_OK) return fp_fail(rc, "%s: layer %d GEMM launch failed", who, l);
    }
    return FP_OK;
}

int fp_surrogate_infer(const fp_surrogate* net, const float* d_x, int q, float* d_y, void* d_work,
                       unsigned long long work_bytes, int* d_err, void* stream) {
    if (!net || !d_x || !d_y || !d_work) return fp_fail(FP_EINVAL, "fp_surrogate_infer: NULL argument");
    if (q < 0) return fp_fail(FP_EINVAL, "fp_surrogate_infer: q=%d", q);
    if (q == 0) return FP_OK;
    if (work_bytes < infer_ws(q, nullptr, nullptr))
        return fp_fail(FP_EINVAL, "fp_surrogate_infer: workspace %llu < %zu bytes", work_bytes,
                       infer_ws(q, nullptr, nullptr));
    if (!d_err) return fp_fail(FP_EINVAL, "fp_surrogate_infer: d_err is required");
    InferWs w;
    infer_ws(q, (unsigned char*)d_work, &w);
    return infer_member(net, d_x, q, d_y, w, d_err, nullptr, (cudaStream_t)stream, "fp_surrogate_infer");
}

// spread[r] = sqrt(sum |y0 - y1|^2) / (2 sqrt(sum |mean|^2))
__global__ void ensemble_spread_kernel(const float* __restrict__ rowacc, int q, float* __restrict__ spread) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= q) return;
    spread[r] = sqrtf(rowacc[2 * r]) / (2.f * fmaxf(sqrtf(rowacc[2 * r + 1]), 1e-30f));
}

int fp_surrogate_infer_ensemble(const fp_surrogate* net0, const fp_surrogate* net1, const float* d_x, int q,
                                float* d_mean, float* d_spread, void* d_work, unsigned long long work_bytes,
                                int* d_err, void* stream) {
    if (!net0 || !net1 || !d_x || !d_mean || !d_spread || !d_work || !d_err)
        return fp_fail(FP_EINVAL, "fp_surrogate_infer_ensemble: NULL argument");
    if (q < 0) return fp_fail(FP_EINVAL, "fp_surrogate_infer_ensemble: q=%d", q);
    if (q == 0) return FP_OK;
    const size_t base = infer_ws(q, nullptr, nullptr), need = base + al256((size_t)q * 2 * sizeof(float));
    if (work_bytes < need)
        return fp_fail(FP_EINVAL, "fp_surrogate_infer_ensemble: workspace %llu < %zu bytes", work_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    InferWs w;
    infer_ws(q, (unsigned char*)d_work, &w);
    float* rowacc = (float*)((unsigned char*)d_work + base);
    if (cudaMemsetAsync(rowacc, 0, (size_t)q * 2 * sizeof(float), st) != cudaSuccess)
        return fp_fail(FP_ECUDA, "fp_surrogate_infer_ensemble: memset");
    int rc = infer_member(net0, d_x, q, d_mean, w, d_err, nullptr, st, "fp_surrogate_infer_ensemble");
    if (rc != FP_OK) return rc;
    rc = infer_member(net1, d_x, q, d_mean, w, d_err, rowacc, st, "fp_surrogate_infer_ensemble");
    if (rc != FP_OK) return rc;
    ensemble_spread_kernel<<<(q + 255) / 256, 256, 0, st>>>(rowacc, q, d_spread);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_surrogate_infer_ensemble: spread kernel");
    return FP_OK;
}

int fp_surrogate_grad(const fp_surrogate_train* t, const float* d_x, const float* d_y, int q, float* d_loss,
                      float* const* d_gW, float* const* d_gb, void* d_work, unsigned long long work_bytes,
                      int* d_err, void* stream) {
    if (!t || !d_x || !d_y || !d_loss || !d_gW || !d_gb || !d_work || !d_err)
        return fp_fail(FP_EINVAL, "fp_surrogate_grad: NULL argument");
    if (q < 8 || q % 8) return fp_fail(FP_EINVAL, "fp_surrogate_grad: q=%d must be a positive multiple of 8", q);
    for (int l = 0; l < FP_SUR_LAYERS; ++l)
        if (!t->net.W[l] || !t->net.b[l] || !d_gW[l] || !d_gb[l] || (l > 0 && !t->WT[l]))
            return fp_fail(FP_EINVAL, "fp_surrogate_grad: layer %d not set", l);
    if (work_bytes < train_ws(q, nullptr, nullptr))
        return fp_fail(FP_EINVAL, "fp_surrogate_grad: workspace %llu < %zu bytes", work_bytes,
                       train_ws(q, nullptr, nullptr));
    cudaStream_t st = (cudaStream_t)stream;
    TrainWs w;
    train_ws(q, (unsigned char*)d_work, &w);
    if (cudaMemsetAsync(d_loss, 0, sizeof(float), st) != cudaSuccess ||
        cudaMemsetAsync(w.x0T, 0, (size_t)FP_SUR_KIN * w.ldt * 2, st) != cudaSuccess)
        return fp_fail(FP_ECUDA, "fp_surrogate_grad: memset");
    const long long tot = (long long)q * FP_SUR_KIN;
    prep_input_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d_x, q, t->net.in_shift, t->net.in_scale,
                                                                       w.x0, w.x0T, w.ldt);
    if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_surrogate_grad: input kernel launch");
    // forward, keeping pre-activations and transposed activations
    const __nv_bfloat16* x = w.x0;
    int rc;
    for (int l = 0; l < FP_SUR_LAYERS - 1; ++l) {
        EpiParams P = epi0(d_err);
        P.bias = t->net.b[l];
        P.out = w.h[l]; P.ldo = FP_SUR_HIDDEN;
        P.outT = w.hT[l]; P.ldt = w.ldt;
        P.outf = w.z[l]; P.ldf = FP_SUR_HIDDEN;
        rc = gemm(EPI_HIDDEN_TRAIN, 256, x, KL[l], t->net.W[l], KL[l], q, NL[l], KL[l], P, st);
        if (rc != FP_OK) return fp_fail(rc, "fp_surrogate_grad: forward layer %d", l);
        x = w.h[l];
    }
    {
        EpiParams P = epi0(d_err);
        P.bias = t->net.b[4];
        P.y = d_y; P.ldy = FP_SUR_OUT;
        P.oshift = t->net.out_shift; P.oscale = t->net.out_scale;
        P.loss = d_loss;
        P.gscale = 2.f / ((float)q * (float)FP_SUR_OUT);
        P.out = w.g4; P.ldo = FP_SUR_OUT;
        P.outT = w.g4T; P.ldt = w.ldt;
        rc = gemm(EPI_OUT_TRAIN, 160, x, KL[4], t->net.W[4], KL[4], q, NL[4], KL[4], P, st);
        if (rc != FP_OK) return fp_fail(rc, "fp_surrogate_grad: output layer");
    }
    // backward
    const __nv_bfloat16* G = w.g4;
    const __nv_bfloat16* GT = w.g4T;
    for (int l = FP_SUR_LAYERS - 1; l >= 0; --l) {
        const __nv_bfloat16* XT = l == 0 ? w.x0T : w.hT[l - 1];
        {   // dW_l [N_l][K_l] = G^T X: A = G^T [N_l][q], B = X^T [K_l][q]
            EpiParams P = epi0(d_err);
            P.outf = d_gW[l]; P.ldf = KL[l];
            rc = gemm(EPI_DW, KL[l] == FP_SUR_KIN ? 64 : 256, GT, w.ldt, XT, w.ldt, NL[l], KL[l], q, P, st);
            if (rc != FP_OK) return fp_fail(rc, "fp_surrogate_grad: dW layer %d", l);
        }
        bias_grad_kernel<<<(NL[l] + 7) / 8, 256, 0, st>>>(GT, w.ldt, q, NL[l], d_gb[l]);
        if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_surrogate_grad: bias kernel");
        if (l == 0) break;
        {   // G_{l-1} = (G W_l) * gelu'(z_{l-1}): A = G [q][N_l], B = W_l^T [K_l][N_l]
            EpiParams P = epi0(d_err);
            P.zin = w.z[l - 1]; P.ldz = FP_SUR_HIDDEN;
            P.out = w.g[l & 1]; P.ldo = FP_SUR_HIDDEN;
            P.outT = w.gT[l & 1]; P.ldt = w.ldt;
            rc = gemm(EPI_DX_GELU, 256, G, NL[l], t->WT[l], NL[l], q, KL[l], NL[l], P, st);
            if (rc != FP_OK) return fp_fail(rc, "fp_surrogate_grad: dX layer %d", l);
            G = w.g[l & 1];
            GT = w.gT[l & 1];
        }
    }
    return FP_OK;
}

int fp_surrogate_adam(const fp_surrogate_train* t, float* const* d_gW, float* const* d_gb, float lr, float beta1,
                      float beta2, float eps, int step, void* stream) {
    if (!t || step < 0) return fp_fail(FP_EINVAL, "fp_surrogate_adam: bad argument");
    if (step > 0 && (!d_gW || !d_gb)) return fp_fail(FP_EINVAL, "fp_surrogate_adam: NULL gradients");
    AdamArgs a;
    a.lr = lr; a.b1 = beta1; a.b2 = beta2; a.eps = eps; a.step = step;
    a.c1 = step > 0 ? 1.f - powf(beta1, (float)step) : 1.f;
    a.c2 = step > 0 ? 1.f - powf(beta2, (float)step) : 1.f;
    cudaStream_t st = (cudaStream_t)stream;
    for (int l = 0; l < FP_SUR_LAYERS; ++l) {
        if (!t->Wm[l] || !t->net.W[l] || (step > 0 && (!t->mW[l] || !t->vW[l] || !t->bm[l] || !t->mb[l] ||
                                                        !t->vb[l] || !d_gW[l] || !d_gb[l])))
            return fp_fail(FP_EINVAL, "fp_surrogate_adam: layer %d not set", l);
        const long long tot = (long long)NL[l] * KL[l] + NL[l];
        adam_layer_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
            t->Wm[l], step > 0 ? d_gW[l] : nullptr, t->mW[l], t->vW[l], t->bm[l], step > 0 ? d_gb[l] : nullptr,
            t->mb[l], t->vb[l], (__nv_bfloat16*)t->net.W[l], l > 0 ? (__nv_bfloat16*)t->WT[l] : nullptr, NL[l],
            KL[l], a);
        if (cudaGetLastError() != cudaSuccess) return fp_fail(FP_ECUDA, "fp_surrogate_adam: launch layer %d", l);
    }
    return FP_OK;
}

}  // extern "C"
