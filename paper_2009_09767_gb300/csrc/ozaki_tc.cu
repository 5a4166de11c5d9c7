// ozaki_tc.cu -- the exact-slice FP64-accurate product (see ozaki.cu for the
// splitting) on the fifth-generation tensor cores: tcgen05.mma with operands
// in shared memory and FP32 accumulators in tensor memory (TMEM).
//
// C = alpha A B^T (+ beta C) from the S bf16 slices of A (m rows) and B
// (n rows).  Every slice pair (a, b) with a + b <= S + 1 gets its own TMEM
// accumulator, so that its sum stays an exact integer in FP32: |s_a s_b| <=
// 2^14, and 1024 products sum to at most 2^24.  Every 1024 k (and at the
// end) the accumulators are read into registers and added, with the pair's
// weight 2^(8 (S + 1 - a - b)), to one 64-bit integer per output.  The
// result is bit for bit that of the mma.sync kernel of ozaki.cu: both form
// the same integers and convert them once.
//
// CTA: 128 threads, output tile 128 x 32 (row i of the tile = TMEM lane i =
// thread i at the drain), S (S + 1) / 2 <= 15 accumulators of 32 columns in
// one 512-column TMEM allocation.  k runs in stages of 64 through two shared
// buffers (cp.async, canonical no-swizzle K-major layout: 8-row x 16-byte
// core matrices, 128 bytes apart along k and 1024 bytes apart along rows);
// thread 0 issues the stage's MMAs (M = 128, N = 32, K = 16) and commits
// them to the buffer's mbarrier, which the loads of the stage two ahead wait
// on.  Every wait is bounded: on expiry the CTA records an error, lets its
// copies land, frees its TMEM and returns.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

constexpr int TBM = 128, TBN = 32, TBK = 64;
constexpr int kDrainK = 1024;                       // exact run of one accumulator
constexpr int kStagesPerDrain = kDrainK / TBK;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitLimit = 1ll << 24;         // try_wait polls before giving up

template <int S>
struct TcSmem {
    static constexpr int A_BYTES = TBM * TBK * 2;    // one slice, 16 KB
    static constexpr int B_BYTES = TBN * TBK * 2;    // 4 KB
    static constexpr int STAGE = S * (A_BYTES + B_BYTES);
    static constexpr int BYTES = 2 * STAGE + 128;    // + mbarriers and the TMEM address
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle, K-major: start, leading byte
// offset (next core matrix along k), stride byte offset (next 8 rows)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N = TBN, M = TBM
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_test(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void cp16(uint32_t saddr, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ int tc_exp(unsigned long long bits) {
    if (bits == 0ull) return 0;
    const int ef = (int)((bits >> 52) & 0x7ff);
    return (ef == 0 ? 1 : ef) - 1022;
}

// byte offset of (row r, 16-byte chunk c along k) in a tile of the canonical layout
__device__ __forceinline__ uint32_t core_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + c * 128 + (r & 7) * 16);
}

template <int S>
__global__ void __launch_bounds__(128, 1)
k_oz_umma(int m, int n, int64_t kpad, int64_t kc, const uint16_t* __restrict__ As,
          const unsigned long long* __restrict__ amaxA, int rowsA_pad,
          const uint16_t* __restrict__ Bs, const unsigned long long* __restrict__ amaxB,
          int rowsB_pad, double alpha, double beta, double* __restrict__ C, int64_t ldc,
          int64_t strideC, int64_t strideSplit, int nsplit, int sym, int* __restrict__ err) {
    constexpr int NP = S * (S + 1) / 2;
    static_assert(NP * TBN <= (int)kTmemCols, "accumulators exceed the TMEM allocation");
    const int i0 = blockIdx.y * TBM, j0 = blockIdx.x * TBN;
    if (sym && j0 + TBN - 1 < i0) return;   // below the diagonal: mirrored from above
    const int b = blockIdx.z / nsplit, split = blockIdx.z % nsplit;
    const int64_t kb = (int64_t)split * kc;
    const int64_t ke = min(kpad, kb + kc);
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    const uint32_t sbase = smem_u32(tc_sm);
    const uint32_t mbar0 = sbase + 2 * TcSmem<S>::STAGE;   // two 8-byte mbarriers
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_sm + 2 * TcSmem<S>::STAGE + 16);
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t sliceA = (int64_t)rowsA_pad * kpad, sliceB = (int64_t)rowsB_pad * kpad;
    const uint16_t* Ab = As + (int64_t)b * S * sliceA + (int64_t)i0 * kpad;
    const uint16_t* Bb = Bs + (int64_t)b * S * sliceB + (int64_t)j0 * kpad;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        mbar_init(mbar0, 1);
        mbar_init(mbar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tmem_slot;

    long long acc[TBN];
#pragma unroll
    for (int c = 0; c < TBN; ++c) acc[c] = 0;

    // stage loads: A slices (TBM rows x TBK) then B slices (TBN rows x TBK),
    // 16-byte chunks; k beyond ke reads as zero
    auto load_stage = [&](int buf, int64_t k0) {
        const uint32_t st = sbase + buf * TcSmem<S>::STAGE;
        constexpr int CA = S * TBM * (TBK / 8), CB = S * TBN * (TBK / 8);
        for (int q = tid; q < CA + CB; q += 128) {
            int sl, r, ch;
            uint32_t dst;
            const uint16_t* src;
            if (q < CA) {
                sl = q / (TBM * (TBK / 8));
                const int rem = q % (TBM * (TBK / 8));
                r = rem / (TBK / 8);
                ch = rem % (TBK / 8);
                dst = st + sl * TcSmem<S>::A_BYTES + core_off(r, ch);
                src = Ab + sl * sliceA + (int64_t)r * kpad + k0 + ch * 8;
            } else {
                const int qq = q - CA;
                sl = qq / (TBN * (TBK / 8));
                const int rem = qq % (TBN * (TBK / 8));
                r = rem / (TBK / 8);
                ch = rem % (TBK / 8);
                dst = st + S * TcSmem<S>::A_BYTES + sl * TcSmem<S>::B_BYTES + core_off(r, ch);
                src = Bb + sl * sliceB + (int64_t)r * kpad + k0 + ch * 8;
            }
            if (k0 + ch * 8 < ke) {
                cp16(dst, src);
            } else {
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(0u), "r"(0u),
                             "r"(0u), "r"(0u));
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    // drain: every accumulator into the 64-bit sums (all 128 threads)
    auto drain = [&]() {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int p = 0;
#pragma unroll 1
        for (int a = 1; a <= S; ++a) {
#pragma unroll 1
            for (int bs = 1; a + bs <= S + 1; ++bs, ++p) {
                uint32_t r[32];
                tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(p * TBN), r);
                const int sh = 8 * (S + 1 - a - bs);
#pragma unroll
                for (int c = 0; c < TBN; ++c)
                    acc[c] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    const int nst = (int)((ke - kb + TBK - 1) / TBK);
    int last = -1;   // last stage whose MMAs were committed
    for (int it = 0; it < nst; ++it) {
        const int buf = it & 1;
        if (it >= 2 && !mbar_wait(mbar0 + 8 * buf, (uint32_t)(((it - 2) >> 1) & 1))) {
            failed = 1;
        }
        __syncthreads();
        if (failed) break;
        load_stage(buf, kb + (int64_t)it * TBK);
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = sbase + buf * TcSmem<S>::STAGE;
            const bool first = (it % kStagesPerDrain) == 0;
            int p = 0;
#pragma unroll 1
            for (int a = 1; a <= S; ++a) {
#pragma unroll 1
                for (int bs = 1; a + bs <= S + 1; ++bs, ++p) {
                    const uint32_t sa = st + (a - 1) * TcSmem<S>::A_BYTES;
                    const uint32_t sb = st + S * TcSmem<S>::A_BYTES + (bs - 1) * TcSmem<S>::B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TBK / 16; ++kk)
                        umma_bf16(tbase + (uint32_t)(p * TBN), umma_desc(sa + kk * 256, 128, 1024),
                                  umma_desc(sb + kk * 256, 128, 1024),
                                  (first && kk == 0) ? 0u : 1u);
                }
            }
            umma_commit(mbar0 + 8 * buf);
        }
        last = it;
        if ((it % kStagesPerDrain) == kStagesPerDrain - 1 || it == nst - 1) {
            if (!mbar_wait(mbar0 + 8 * buf, (uint32_t)((it >> 1) & 1))) failed = 1;
            __syncthreads();
            if (failed) break;
            drain();
            __syncthreads();
        }
    }
    const bool ok = !failed;
    __syncthreads();
    // on a failed wait, give the last committed MMAs (bounded) time to land
    // before their TMEM is freed
    if (!ok && last >= 0) mbar_wait(mbar0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1));
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(kTmemCols));
    }
    if (!ok) {
        if (tid == 0 && err) atomicExch(err, 1);
        return;
    }
    // epilogue: row i = i0 + tid, columns j0 .. j0 + 31
    double* Cb = C + (int64_t)b * strideC + (int64_t)split * strideSplit;
    const int i = i0 + tid;
    if (i >= m) return;
    const int ei = tc_exp(amaxA[(int64_t)b * rowsA_pad + i]);
#pragma unroll
    for (int c = 0; c < TBN; ++c) {
        const int j = j0 + c;
        if (j >= n || (sym && j < i)) continue;
        const int ej = tc_exp(amaxB[(int64_t)b * rowsB_pad + j]);
        double v = alpha * ldexp((double)acc[c], ei + ej - 14 - 8 * (S - 1));
        double* cp = Cb + (int64_t)i * ldc + j;
        if (beta != 0.0) v += beta * *cp;
        *cp = v;
        if (sym && j != i) Cb[(int64_t)j * ldc + i] = v;
    }
}

template <int S>
cudaError_t umma_gemm_t(int nb, int m, int n, int64_t kpad, int nsplit, const OzOperand& A,
                        const OzOperand& B, double alpha, double beta, double* C, int64_t ldc,
                        int64_t strideC, int64_t strideSplit, int sym, int* err, cudaStream_t s) {
    constexpr int smem = TcSmem<S>::BYTES;
    RK_CUDA_TRY(cudaFuncSetAttribute(k_oz_umma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int64_t kc = round_up(ceil_div(kpad, nsplit), 32);
    dim3 grid((unsigned)ceil_div(n, TBN), (unsigned)ceil_div(m, TBM), (unsigned)(nb * nsplit));
    k_oz_umma<S><<<grid, 128, smem, s>>>(m, n, kpad, kc, A.slices, A.amax, A.rows_pad, B.slices,
                                         B.amax, B.rows_pad, alpha, beta, C, ldc, strideC,
                                         strideSplit, nsplit, sym, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_oz_gemm_tc(int nb, int m, int n, const OzOperand& A, const OzOperand& B,
                              double alpha, double beta, double* C, int64_t ldc, int64_t strideC,
                              int sym, cudaStream_t s, int nsplit, int64_t strideSplit, int* err) {
    if (A.S != B.S || A.kpad != B.kpad || m > A.rows_pad || n > B.rows_pad || nsplit < 1)
        return cudaErrorInvalidValue;
    if (A.rows_pad % TBM != 0 || B.rows_pad % TBN != 0 || A.kpad % 32 != 0)
        return cudaErrorInvalidValue;
    if (sym && m != n) return cudaErrorInvalidValue;
    if (nb <= 0 || m <= 0 || n <= 0) return cudaSuccess;
    if (A.S == 3)
        return umma_gemm_t<3>(nb, m, n, A.kpad, nsplit, A, B, alpha, beta, C, ldc, strideC,
                              strideSplit, sym, err, s);
    return umma_gemm_t<5>(nb, m, n, A.kpad, nsplit, A, B, alpha, beta, C, ldc, strideC, strideSplit,
                          sym, err, s);
}

}  // namespace rk
