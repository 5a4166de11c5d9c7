// ozaki_tc.cu -- the exact-slice FP64-accurate product (see ozaki.cu for the
// splitting) on the fifth-generation tensor cores: operands brought into
// shared memory by the tensor memory accelerator (cp.async.bulk.tensor, 64-
// byte swizzle), tcgen05.mma with FP32 accumulators in tensor memory (TMEM).
//
// C = alpha A B^T (+ beta C) from the S bf16 slices of A (m rows) and B
// (n rows).  The slice pairs (a, b) with a + b <= S + 1 of one weight
// w = a + b share a TMEM accumulator: w - 1 <= S pairs, each product
// |s_a s_b| <= 2^14, so a run of up to 1024 / S in k sums to at most 2^24 and
// stays an exact integer in FP32.  After every such run (and at the end) the
// S accumulators are read into registers and added, with the weight
// 2^(8 (S + 1 - w)), to one 64-bit integer per output.  The result is bit
// for bit that of the mma.sync kernel of ozaki.cu: both form the same
// integers and convert them once.
//
// CTA: 128 threads, output tile 128 x 32 (row i of the tile = TMEM lane i =
// thread i at the drain), S accumulators of 32 columns in a 256-column TMEM
// allocation, k in stages of 32 through NBUF shared buffers of about 108 KB
// in all, so that two CTAs share an SM: one's drain and epilogue overlap
// the other's copies and MMAs (a 128 x 64 tile, one CTA per SM with three
// stages in flight, was 12% slower on the refinement's products).  Warp 0 runs
// the pipeline (lane 0 issues): each stage's tensor copies (one per slice
// and operand, completion counted in bytes on the buffer's "full" mbarrier)
// and, once they have landed, the stage's MMAs (M = 128, N = 32, K = 16),
// committed to the buffer's "empty" mbarrier before the buffer is refilled;
// the other warps wait for the drain.  Shared tiles are K-major with the
// 64-byte swizzle: rows of 32 bf16, 8-row atoms of 512 bytes; the second
// MMA of a stage starts 32 bytes into the rows.  Every wait is bounded: on expiry the CTA records an
// error, lets what it issued land (bounded), frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

constexpr int TBM = 128, TBN = 32, TBK = 32;
constexpr uint32_t kTmemCols = 256;
constexpr long long kWaitCycles = 1ll << 31;        // ~1 s of SM clock before a wait gives up

template <int S>
struct TcSmem {
    static constexpr int A_BYTES = TBM * TBK * 2;    // one slice tile, 8 KB
    static constexpr int B_BYTES = TBN * TBK * 2;    // 2 KB
    static constexpr int STAGE = S * (A_BYTES + B_BYTES);
    static constexpr int NBUF = (108 * 1024) / STAGE;  // two CTAs per SM
    static constexpr int BAR = NBUF * STAGE;         // barriers after the buffers
    static constexpr int BYTES = BAR + 256 + 1024;   // + barriers, TMEM slot, alignment slack
    // exact run of an accumulator: S pairs x k x 2^14 <= 2^24
    static constexpr int STAGES_PER_DRAIN = (1024 / S) / TBK;
    static_assert(S * TBN <= (int)kTmemCols, "accumulators fit the allocation");
    static_assert(2 * (BYTES + 1024) <= 228 * 1024, "two CTAs per SM");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row atoms
// 512 bytes apart (stride byte offset); the leading byte offset is unused
// for this layout (encoded 1)
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                     // leading byte offset (16 B, unused)
    d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version of this architecture
    d |= (uint64_t)4 << 61;                     // layout: 64-byte swizzle
    return d;
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
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

// bounded wait for the phase of the given parity; false when about a second
// of SM clock passed or (when given) the CTA's failure flag was raised
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          const volatile int* failed = nullptr) {
    const long long t0 = clock64();
    for (unsigned i = 0;; ++i) {
        if (mbar_test(mbar, parity)) return true;
        if ((i & 63) == 63) {
            if (clock64() - t0 > kWaitCycles) return false;
            if (failed && *failed) return false;
        }
    }
}

// 3-d tensor copy global -> shared (coordinates k, row, slice), completion
// counted on mbar
__device__ __forceinline__ void tma_load(uint32_t sdst, const CUtensorMap* map, int x, int y, int z,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(sdst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
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

template <int S>
__global__ void __launch_bounds__(128, 2)
k_oz_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m,
          int n, int64_t kpad, int64_t kc, const unsigned long long* __restrict__ amaxA,
          int rowsA_pad, const unsigned long long* __restrict__ amaxB, int rowsB_pad,
          double alpha, double beta, double* __restrict__ C, int64_t ldc, int64_t strideC,
          int64_t strideSplit, int nsplit, int sym, int* __restrict__ err) {
    using L = TcSmem<S>;
    constexpr int NB = L::NBUF;
    const int i0 = blockIdx.y * TBM, j0 = blockIdx.x * TBN;
    if (sym && j0 + TBN - 1 < i0) return;   // below the diagonal: mirrored from above
    const int b = blockIdx.z / nsplit, split = blockIdx.z % nsplit;
    const int64_t kb = (int64_t)split * kc;
    const int64_t ke = min(kpad, kb + kc);
    extern __shared__ unsigned char tc_sm[];
    const uint32_t sraw = smem_u32(tc_sm);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;          // swizzle atoms want 1024-byte alignment
    const uint32_t full0 = sbase + L::BAR;                     // NB "full" mbarriers
    const uint32_t empty0 = full0 + 8 * NB;                    // NB "empty" mbarriers
    const uint32_t drainb = empty0 + 8 * NB;                   // drain mbarrier
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tc_sm + (drainb + 8 - sraw));
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        failed = 0;
        for (int q = 0; q < NB; ++q) {
            mbar_init(full0 + 8 * q, 1);
            mbar_init(empty0 + 8 * q, 1);
        }
        mbar_init(drainb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tmem_slot;

    long long acc[TBN];
#pragma unroll
    for (int c = 0; c < TBN; ++c) acc[c] = 0;

    const int nst = (int)((ke - kb + TBK - 1) / TBK);
    int issued = 0;        // stages whose copies thread 0 has issued
    int committed = -1;    // last stage whose MMAs thread 0 has committed

    // thread 0: the copies of stage st into buffer st % NB
    auto issue_loads = [&](int st) {
        const int buf = st % NB;
        const uint32_t sb = sbase + buf * L::STAGE;
        const uint32_t fb = full0 + 8 * buf;
        mbar_expect_tx(fb, (uint32_t)L::STAGE);
        const int x = (int)(kb + (int64_t)st * TBK);
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            tma_load(sb + sl * L::A_BYTES, &tmA, x, i0, b * S + sl, fb);
            tma_load(sb + S * L::A_BYTES + sl * L::B_BYTES, &tmB, x, j0, b * S + sl, fb);
        }
    };

    int period = 0;
    const int lane = tid & 31;
    for (int p0 = 0; p0 < nst; p0 += L::STAGES_PER_DRAIN, ++period) {
        const int p1 = min(nst, p0 + L::STAGES_PER_DRAIN);
        // warp 0 runs the copy/MMA loop with uniform control flow (every lane
        // waits, lane 0 issues); warps 1..3 go straight to the drain wait
        if (warp == 0 && !failed) {
            if (lane == 0)
                for (int st = p0; st < min(p1, p0 + NB); ++st) issue_loads(st);
            issued = min(p1, p0 + NB);
            bool ok = true;
            for (int it = p0; it < p1; ++it) {
                const int buf = it % NB;
                const uint32_t par = (uint32_t)((it / NB) & 1);
                ok = __all_sync(0xffffffffu, mbar_wait(full0 + 8 * buf, par));
                if (!ok) break;
                if (lane == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sb = sbase + buf * L::STAGE;
                    // descriptors of slice 1 at k = 0; a slice and a 16-k step move
                    // only the start-address field (16-byte units, no carry:
                    // shared addresses stay below 2^18)
                    const uint64_t dA = umma_desc_sw64(sb);
                    const uint64_t dB = umma_desc_sw64(sb + S * L::A_BYTES);
                    // the run's first MMA into accumulator w - 2 (pair (1, w - 1),
                    // k = 0 of its first stage) overwrites it
                    const uint32_t first = it == p0 ? 0u : 1u;
#pragma unroll
                    for (int a = 1; a <= S; ++a) {
#pragma unroll
                        for (int bs = 1; a + bs <= S + 1; ++bs) {
                            const int q = a + bs - 2;
#pragma unroll
                            for (int kk = 0; kk < TBK / 16; ++kk)
                                umma_bf16(tbase + (uint32_t)(q * TBN),
                                          dA + (uint64_t)(((a - 1) * L::A_BYTES + kk * 32) >> 4),
                                          dB + (uint64_t)(((bs - 1) * L::B_BYTES + kk * 32) >> 4),
                                          (kk == 0 && a == 1) ? first : 1u);
                        }
                    }
                    umma_commit(empty0 + 8 * buf);
                }
                __syncwarp();
                committed = it;
                if (it + NB < p1) {
                    // the buffer is refilled once the MMAs reading it are done
                    ok = __all_sync(0xffffffffu, mbar_wait(empty0 + 8 * buf, par));
                    if (!ok) break;
                    if (lane == 0) issue_loads(it + NB);
                    __syncwarp();
                    issued = it + NB + 1;
                }
            }
            if (!ok) {
                if (lane == 0) failed = 1;
            } else if (lane == 0) {
                umma_commit(drainb);
            }
            __syncwarp();
        }
        // drain: every thread, once the period's MMAs are done
        if (!mbar_wait(drainb, (uint32_t)(period & 1), &failed)) failed = 1;
        __syncthreads();
        if (failed) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {
#pragma unroll 1
            for (int q = 0; q < S; ++q) {            // weight w = q + 2
                const int sh = 8 * (S - 1 - q);
#pragma unroll
                for (int h = 0; h < TBN / 32; ++h) {
                    uint32_t r[32];
                    tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * TBN + h * 32), r);
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        acc[h * 32 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    const bool ok = !failed;
    if (!ok && tid == 0) {   // (issued and committed are warp 0's, uniform across it)
        // let what was issued land before the shared memory and TMEM go away
        for (int st = committed + 1; st < issued; ++st)
            mbar_wait(full0 + 8 * (st % NB), (uint32_t)((st / NB) & 1));
        if (committed >= 0)
            mbar_wait(empty0 + 8 * (committed % NB), (uint32_t)((committed / NB) & 1));
    }
    __syncthreads();
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

// cuTensorMapEncodeTiled from the driver, looked up once
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
    static std::once_flag once;
    static EncodeFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// the slices of an operand as a 3-d tensor (k, row, batch x slice) of
// 16-bit elements; boxes of 32 k x box_rows rows, 64-byte swizzle
cudaError_t slice_map(CUtensorMap* map, const OzOperand& op, int nb, int box_rows) {
    EncodeFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)op.kpad, (cuuint64_t)op.rows_pad,
                                (cuuint64_t)nb * (cuuint64_t)op.S};
    const cuuint64_t strides[2] = {(cuuint64_t)op.kpad * 2,
                                   (cuuint64_t)op.rows_pad * (cuuint64_t)op.kpad * 2};
    const cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, op.slices, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S>
cudaError_t umma_gemm_t(int nb, int m, int n, int64_t kpad, int nsplit, const OzOperand& A,
                        const OzOperand& B, double alpha, double beta, double* C, int64_t ldc,
                        int64_t strideC, int64_t strideSplit, int sym, int* err, cudaStream_t s) {
    constexpr int smem = TcSmem<S>::BYTES;
    CUtensorMap ta, tb;
    RK_CUDA_TRY(slice_map(&ta, A, nb, TBM));
    RK_CUDA_TRY(slice_map(&tb, B, nb, TBN));
    RK_CUDA_TRY(cudaFuncSetAttribute(k_oz_umma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // split chunks on stage boundaries: a tensor copy past a chunk's end would
    // read the next chunk (past kpad it reads zeros)
    const int64_t kc = round_up(ceil_div(kpad, nsplit), TBK);
    dim3 grid((unsigned)ceil_div(n, TBN), (unsigned)ceil_div(m, TBM), (unsigned)(nb * nsplit));
    k_oz_umma<S><<<grid, 128, smem, s>>>(ta, tb, m, n, kpad, kc, A.amax, A.rows_pad, B.amax,
                                         B.rows_pad, alpha, beta, C, ldc, strideC, strideSplit,
                                         nsplit, sym, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_oz_gemm_tc(int nb, int m, int n, const OzOperand& A, const OzOperand& B,
                              double alpha, double beta, double* C, int64_t ldc, int64_t strideC,
                              int sym, cudaStream_t s, int nsplit, int64_t strideSplit, int* err) {
    if (A.S != B.S || A.kpad != B.kpad || m > A.rows_pad || n > B.rows_pad || nsplit < 1)
        return cudaErrorInvalidValue;
    if (A.rows_pad % TBM != 0 || B.rows_pad % TBN != 0 || A.kpad % TBK != 0)
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
