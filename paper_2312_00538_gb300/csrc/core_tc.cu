// Woodbury core of the low-rank preconditioner on the tensor cores with FP64 accuracy
// (arXiv 2312.00538, Sec. 5: M = I + L^T Theta^{-1} L in the Woodbury inverse of
// Theta + Y L L^T Y).
//
// M = I + A^T A with A = Theta^{-1/2} L (n x r). The tensor cores multiply bf16 operands into an
// FP32 accumulator, so A is first split into exact integer slices (the error-free splitting of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//   column a of A is scaled by 2^-E_a so that every entry lies in (-1, 1), and
//   x = q_0 2^-w + q_1 2^-2w + ... + q_{S-1} 2^-Sw + rest,  q_s = rint(residual 2^{w(s+1)}),
// with integers |q_s| <= 2^w (w = 6: exact in bf16) and |rest| <= 2^{-wS-1} (S = 9: 2^-55).
// Then A^T A = sum over u of 2^{E_a + E_b - w(u + 2)} I_u with the integer matrices
//   I_u = sum_{s + t = u} Q_s^T Q_t   (u < S; the terms with s + t >= S are below FP64 rounding).
// Every product of two slices is an integer of magnitude <= 2^{2w} = 2^12, so a sum over 4096
// rows is an integer below 2^24 and the FP32 accumulator holds it exactly. Each CTA therefore
// accumulates Q_s^T Q_t over one block of 4096 rows on the tensor cores (tcgen05.mma kind::f16, bf16 inputs, M = 128 rows a, N = 128 or 256 columns b,
// FP32 accumulator in tensor memory) and adds the exact chunk sums into FP64 accumulators of I_u
// with atomics. The totals stay integers below 2^53, so FP64 addition is exact in any order and
// the result does not depend on the order in which CTAs finish. A last kernel scales and sums the
// I_u in FP64 in a fixed order (smallest terms first) and adds the identity.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "lowrank_internal.h"
#include "tcgen05.cuh"

namespace anova {
anova_status fail(anova_status st, const std::string &msg);
anova_status cuda_fail(cudaError_t e, const char *what);

namespace {

constexpr int kW = 6;            // bits per slice
constexpr int kS = 9;            // slices
constexpr int kChunk = 4096;     // rows per exact FP32 accumulation (one CTA)
constexpr int kKS = 32;          // rows per shared-memory stage (two K = 16 products)
constexpr int kNS = 4;           // stage slots (three stages in flight while one is multiplied)
constexpr int kMRows = 128;      // MMA M: rows a per CTA
constexpr uint32_t kMaxPolls = 1u << 22;

// ---------------------------------------------------------------- scales and column exponents
// s_i = sqrt(1 / theta_i) (FP64, and rounded to FP32 for the column maxima), so that
// A(i, a) = L(i, a) s_i.
__global__ void k_core_rowscale(const double *__restrict__ itheta, long long n, double *__restrict__ srow,
                                float *__restrict__ srow32) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = sqrt(itheta[i]);
        srow[i] = v;
        srow32[i] = (float)v;
    }
}

// cmax[a] >= max_i |A(i, a)| (bits of a non-negative float, so an integer atomic max finds it):
// FP32 products, whose relative error (<= 2^-23 with the rounding of s_i) the exponent margin in
// col_exponent covers. Grid (row chunks, columns).
__global__ void __launch_bounds__(256) k_core_colmax(const float *__restrict__ L, const float *__restrict__ srow32,
                                                     long long n, unsigned *__restrict__ cmax) {
    __shared__ float red[8];
    const int a = blockIdx.y;
    float mx = 0.0f;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        mx = fmaxf(mx, fabsf(L[(long long)a * n + i] * srow32[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
        atomicMax(&cmax[a], __float_as_uint(m));
    }
}

// E_a with max_i |A(i, a)| < 2^E_a, from the FP32 maximum enlarged by 2^-20 (0 for a zero column)
__device__ __forceinline__ int col_exponent(unsigned mbits) {
    const float m = __uint_as_float(mbits);
    if (!(m > 0.0f)) return 0;
    const unsigned ub = __float_as_uint(m * (1.0f + 0x1p-20f));
    return (int)((ub >> 23) & 0xFF) - 127 + 1;
}

// ---------------------------------------------------------------- slices
// Q[s][a][i] (bf16, rows a of np entries): the digits of |A(i, a)| 2^-E_a in base 2^6 with the sign
// of A: X = floor(|A| 2^{54 - E_a}) < 2^54 holds 54 fractional bits and
// q_s = sign * (bits 54 - 6 (s + 1) .. 53 - 6 s of X), so |q_s| <= 63 and
// |A| 2^-E_a = sum_s |q_s| 2^{-6 (s + 1)} + rest, 0 <= rest < 2^-54. A is the exact product of the
// FP32 panel entry and the FP64 scale, formed as a 77-bit integer product of the two significands
// (integer operations only: GB300's FP64 pipe is slow). Zero for rows a >= r and entries i >= n.
__global__ void __launch_bounds__(256) k_core_slice(const float *__restrict__ L, const double *__restrict__ srow,
                                                    long long n, long long np, int r, int RP,
                                                    const unsigned *__restrict__ cmax,
                                                    __nv_bfloat16 *__restrict__ Q) {
    const int a = blockIdx.y;
    const int E = a < r ? col_exponent(cmax[a]) : 0;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < np; i += (long long)gridDim.x * 256) {
        unsigned long long X = 0;
        bool neg = false;
        if (a < r && i < n) {
            const unsigned lb = __float_as_uint(L[(long long)a * n + i]);
            const unsigned long long sb = (unsigned long long)__double_as_longlong(srow[i]);
            const int el = (int)((lb >> 23) & 0xFF), es = (int)((sb >> 52) & 0x7FF);
            neg = (lb >> 31) != 0;
            if (el != 0 && es != 0) {  // normal numbers (subnormal entries lie far below 2^-54 of the column)
                const unsigned long long ml = (lb & 0x7FFFFFu) | 0x800000u;                    // 24 bits
                const unsigned long long ms = (sb & 0xFFFFFFFFFFFFFull) | (1ull << 52);       // 53 bits
                const unsigned long long lo = ml * ms, hi = __umul64hi(ml, ms);             // 77-bit product
                // |A| = P 2^{(el - 127 - 23) + (es - 1023 - 52)}, X = P 2^{that + 54 - E}
                const int sh = -((el - 150) + (es - 1075) + 54 - E);  // right shift of P (>= 23: X < 2^54)
                if (sh >= 128) X = 0;
                else if (sh >= 64) X = hi >> (sh - 64);
                else if (sh > 0) X = (hi << (64 - sh)) | (lo >> sh);
                else X = lo;  // sh <= 0 cannot occur while |A| < 2^E
            }
        }
#pragma unroll
        for (int s = 0; s < kS; ++s) {
            const int d = (int)((X >> (54 - kW * (s + 1))) & ((1ull << kW) - 1));
            Q[((long long)s * RP + a) * np + i] = __int2bfloat16_rn(neg ? -d : d);
        }
    }
}

// ---------------------------------------------------------------- exact slice products
struct CoreMmaArgs {
    const __nv_bfloat16 *Q;  // [kS][RP][np]
    long long np;
    int r;
    const int4 *work;        // per CTA: {s, t, row block, 0} with s <= t, s + t < kS
    double *I;               // [kS][RP][RP] integer accumulators (upper triangle, a <= b < r)
    int *status;             // bit 0: a bounded wait ran out
};

// RP = 128 or 256 rows a (= columns b); the CTA holds all of them: RP / 128 accumulators of
// 128 x RP in tensor memory (at most 512 columns)
template <int RP>
struct CoreCfg {
    static constexpr int MB = RP / kMRows;            // MMA row blocks
    static constexpr uint32_t T_BYTES = RP * kKS * 2; // one operand tile (RP rows x kKS)
    static constexpr uint32_t STAGE = 2 * T_BYTES;    // A (slice s) and B (slice t)
    static constexpr uint32_t MBAR = kNS * STAGE, SLOT = MBAR + 8 * kNS;
    static constexpr size_t smem = SLOT + 16;
    static constexpr uint32_t TMEM_COLS = MB * RP;
    // bf16 operands, K-major, no swizzle: core matrices of 8 rows x 16 bytes (8 bf16);
    // element (row, k) of a tile at (row / 8) * SBO + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2
    static constexpr uint32_t LBO = 128, SBO = 128 * (kKS / 8);
    // kind::f16: FP32 accumulator (bit 4), A and B bf16 (bits 7, 10), K-major, N >> 3, M >> 4
    static constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(RP >> 3) << 17) |
                                      ((uint32_t)(kMRows >> 4) << 24);
    static_assert(TMEM_COLS <= 512, "accumulators fit the tensor memory of an SM");
};

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// P = Q_s^T Q_t over rows k0 .. k0 + kChunk - 1 (exact in FP32), added to I_{s + t}: for s < t the
// pair (t, s) gives P^T, so every entry P(a, b) goes to the upper-triangle slot (min, max), the
// diagonal twice; for s = t, P is symmetric and only its upper triangle is added.
template <int RP>
__global__ void __launch_bounds__(128, 1) k_core_mma(CoreMmaArgs a) {
    using C = CoreCfg<RP>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + C::MBAR);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem_raw + C::SLOT);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int4 wk = a.work[blockIdx.x];
    const int s_a = wk.x, s_b = wk.y, u = wk.x + wk.y;
    const bool same = s_a == s_b;                               // A tile = B tile
    const long long k0 = (long long)wk.z * kChunk;
    const int nst = (int)((min(a.np, k0 + kChunk) - k0) / kKS);  // np is a multiple of kKS

    if (warp == 0) tc::tmem_alloc(slot, C::TMEM_COLS);
    if (t == 0) {
        for (int q = 0; q < kNS; ++q) tc::mbar_init(&mbar[q], 1);
        tc::mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t sbase = tc::smem_u32(smem_raw);

    // stage j: rows k0 + kKS j .. of slice s_b (B tile) and, unless s_a = s_b, of slice s_a (A tile)
    auto load_stage = [&](int j, int sl) {
        const long long ki = k0 + (long long)j * kKS;
        const __nv_bfloat16 *qb = a.Q + (long long)s_b * RP * a.np + ki;
        const __nv_bfloat16 *qa = a.Q + (long long)s_a * RP * a.np + ki;
        const uint32_t sb = sbase + sl * C::STAGE, sa = sb + C::T_BYTES;
        constexpr int PC = kKS / 8;  // 16-byte pieces per row
        const int pieces = (same ? 1 : 2) * RP * PC;
        for (int idx = t; idx < pieces; idx += 128) {
            const int tile = idx / (RP * PC), e = idx % (RP * PC);
            const int row = e / PC, pc = e % PC;
            const uint32_t off = (row >> 3) * C::SBO + pc * C::LBO + (row & 7) * 16;
            cp_async16((tile ? sa : sb) + off, (tile ? qa : qb) + (long long)row * a.np + pc * 8);
        }
    };

    bool failed = false;
    int last = -1;  // the last stage whose products were committed (they complete in order)
#pragma unroll
    for (int j = 0; j < kNS - 1; ++j) {
        if (j < nst) load_stage(j, j);
        cp_async_commit();
    }
    for (int it = 0; it < nst; ++it) {
        const int sl = it % kNS;
        cp_async_wait<kNS - 2>();
        tc::fence_proxy_async();
        if (__syncthreads_or(failed)) break;
        if (t == 0) {
            tc::fence_after_sync();
            const uint32_t sb = sbase + sl * C::STAGE, sa = same ? sb : sb + C::T_BYTES;
#pragma unroll
            for (int ks = 0; ks < kKS / 16; ++ks) {
                const uint64_t bd = tc::smem_desc(sb + ks * 256, C::LBO, C::SBO);
#pragma unroll
                for (int mb = 0; mb < C::MB; ++mb) {
                    const uint64_t ad = tc::smem_desc(sa + mb * (kMRows / 8) * C::SBO + ks * 256, C::LBO, C::SBO);
                    mma_bf16(tmem + (uint32_t)(mb * RP), ad, bd, C::idesc, it > 0 || ks > 0);
                }
            }
            tc::mma_commit(&mbar[sl]);
        }
        last = it;
        // refill the slot of stage it - 1 with stage it + kNS - 1 once its products have read it
        // (the barrier of a slot completes once per stage that used it: stage j has parity j / kNS)
        const int nx = it + kNS - 1;
        if (nx < nst) {
            if (it >= 1 && !tc::mbar_wait_bounded(&mbar[(it - 1) % kNS], (uint32_t)(((it - 1) / kNS) & 1), kMaxPolls))
                failed = true;
            if (!failed) load_stage(nx, nx % kNS);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    // the last committed stage's barrier covers every product before the accumulators are read
    const bool ok = !__syncthreads_or(failed);
    bool done = last >= 0 && tc::mbar_wait_bounded(&mbar[last % kNS], (uint32_t)((last / kNS) & 1), kMaxPolls);
    done = __syncthreads_and(done && ok);
    if (done) {
        tc::fence_after_sync();
        double *Iu = a.I + (long long)u * RP * RP;
#pragma unroll 1
        for (int mb = 0; mb < C::MB; ++mb) {
            const int arow = mb * kMRows + warp * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < RP; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mb * RP + c0), v);
                if (arow < a.r) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int b = c0 + j;
                        if (b >= a.r || v[j] == 0.0f) continue;
                        if (same) {
                            if (b >= arow) atomicAdd(&Iu[(long long)arow * RP + b], (double)v[j]);
                        } else {
                            const int lo = min(arow, b), hi = max(arow, b);
                            atomicAdd(&Iu[(long long)lo * RP + hi], (b == arow ? 2.0 : 1.0) * (double)v[j]);
                        }
                    }
                }
            }
        }
    } else if (t == 0) {
        atomicOr(a.status, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// M(a, b) = [a == b] + sum_{u = S-1 .. 0} 2^{E_a + E_b - w(u + 2)} I_u(a, b), symmetric, row-major.
__global__ void k_core_assemble(const double *__restrict__ I, const unsigned *__restrict__ cmax, int r,
                                int RP, double *__restrict__ M) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)r * r;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / r), b = (int)(e % r);
        if (b < a) continue;
        double s = 0.0;
        for (int u = kS - 1; u >= 0; --u)
            s += ldexp(I[((long long)u * RP + a) * RP + b], col_exponent(cmax[a]) + col_exponent(cmax[b]) - kW * (u + 2));
        if (a == b) s += 1.0;
        M[(long long)a * r + b] = s;
        M[(long long)b * r + a] = s;
    }
}

}  // namespace

bool core_tc_supported(const lowrank *lr) { return lr->rank >= 1 && lr->rank <= 256; }

// Allocates the slices, the integer accumulators and the work list once per preconditioner.
static anova_status core_tc_prepare(lowrank *lr) {
    if (lr->tc_Q) return ANOVA_OK;
    const long long n = lr->n;
    const int r = lr->rank;
    lr->tc_np = (n + kKS - 1) / kKS * kKS;
    lr->tc_RP = r <= 128 ? 128 : 256;
    const int RP = lr->tc_RP;
    // one CTA per slice pair s <= t with s + t < kS (25 pairs; Q_t^T Q_s is the transpose of
    // Q_s^T Q_t) and block of kChunk rows; the pairs of one row block are consecutive, so that CTAs
    // running together share that block of every slice in L2
    std::vector<int4> work;
    const int blocks = (int)((lr->tc_np + kChunk - 1) / kChunk);
    for (int c = 0; c < blocks; ++c)
        for (int sa = 0; sa < kS; ++sa)
            for (int sb = sa; sa + sb < kS; ++sb) work.push_back(make_int4(sa, sb, c, 0));
    lr->tc_nwork = (int)work.size();
    cudaError_t e;
    if ((e = cudaMalloc(&lr->tc_Q, sizeof(__nv_bfloat16) * (size_t)kS * RP * lr->tc_np)) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_I, sizeof(double) * (size_t)kS * RP * RP)) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_cmax, sizeof(unsigned) * RP)) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_srow, sizeof(double) * n)) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_srow32, sizeof(float) * n)) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_work, sizeof(int4) * work.size())) != cudaSuccess ||
        (e = cudaMalloc(&lr->tc_status, sizeof(int))) != cudaSuccess)
        return fail(ANOVA_ERR_OOM, "low-rank tensor-core workspace allocation failed");
    cudaStream_t st = lr->plan->stream;
    ANOVA_CUDA_TRY(cudaMemcpyAsync(lr->tc_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice, st));
    ANOVA_CUDA_TRY(cudaMemsetAsync(lr->tc_status, 0, sizeof(int), st));
    return ANOVA_OK;
}

// M = I + L^T diag(itheta) L into lr->M (row-major r x r, symmetric), on the tensor cores.
anova_status core_tc(lowrank *lr) {
    anova_status s = core_tc_prepare(lr);
    if (s != ANOVA_OK) return s;
    cudaStream_t st = lr->plan->stream;
    const long long n = lr->n;
    const int r = lr->rank, RP = lr->tc_RP;
    k_core_rowscale<<<(int)std::min<long long>((n + 255) / 256, 1024), 256, 0, st>>>(lr->itheta, n, lr->tc_srow,
                                                                                      lr->tc_srow32);
    ANOVA_CUDA_TRY(cudaMemsetAsync(lr->tc_cmax, 0, sizeof(unsigned) * RP, st));
    {
        const int chunks = (int)std::min<long long>((n + 4095) / 4096, 32);
        k_core_colmax<<<dim3(chunks, r), 256, 0, st>>>(lr->L32, lr->tc_srow32, n, lr->tc_cmax);
        const long long blocks = std::min<long long>((lr->tc_np + 255) / 256, 64);
        k_core_slice<<<dim3((unsigned)blocks, RP), 256, 0, st>>>(lr->L32, lr->tc_srow, n, lr->tc_np, r, RP, lr->tc_cmax,
                                                               (__nv_bfloat16 *)lr->tc_Q);
    }
    ANOVA_CUDA_TRY(cudaGetLastError());
    ANOVA_CUDA_TRY(cudaMemsetAsync(lr->tc_I, 0, sizeof(double) * (size_t)kS * RP * RP, st));
    CoreMmaArgs ma;
    ma.Q = (const __nv_bfloat16 *)lr->tc_Q;
    ma.np = lr->tc_np;
    ma.r = r;
    ma.work = (const int4 *)lr->tc_work;
    ma.I = lr->tc_I;
    ma.status = lr->tc_status;
    if (RP == 128) {
        static const cudaError_t attr =
            cudaFuncSetAttribute(k_core_mma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CoreCfg<128>::smem);
        if (attr != cudaSuccess) return cuda_fail(attr, "cudaFuncSetAttribute");
        k_core_mma<128><<<lr->tc_nwork, 128, CoreCfg<128>::smem, st>>>(ma);
    } else {
        static const cudaError_t attr =
            cudaFuncSetAttribute(k_core_mma<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CoreCfg<256>::smem);
        if (attr != cudaSuccess) return cuda_fail(attr, "cudaFuncSetAttribute");
        k_core_mma<256><<<lr->tc_nwork, 128, CoreCfg<256>::smem, st>>>(ma);
    }
    ANOVA_CUDA_TRY(cudaGetLastError());
    k_core_assemble<<<(int)std::min<long long>(((long long)r * r + 255) / 256, 1024), 256, 0, st>>>(lr->tc_I, lr->tc_cmax,
                                                                                                    r, RP, lr->M);
    ANOVA_CUDA_TRY(cudaGetLastError());
    return ANOVA_OK;
}

}  // namespace anova
