// ozaki.cu -- FP64-accurate products on the bf16 tensor cores.
//
// The mixed-precision mode refines FP32 eigenbases with FP64-accurate
// products (R = I - X X^T, S = X G X^T, the proxy cross product P P^T of
// Eq. 3).  This part's FP64 pipes run at a small fraction of its tensor
// rate, so these products are formed by error-free splitting (Ozaki et al.,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59,
// 2012), in a fixed-point form:
//
//  * every row r of an operand (rows x k, the product is C = A B^T) is scaled
//    by 2^-e_r, e_r the smallest power with |x| < 2^e_r over the row, and cut
//    into S signed 8-bit slices:  x 2^(7-e_r) = s_1 + s_2 2^-8 + ... +
//    s_S 2^(-8(S-1)) + remainder, |s_q| <= 128, |remainder| <= 2^(-8(S-1)-1).
//    Each slice is an integer, exact in bf16;
//  * a slice pair (a, b) contributes 2^(e_i+e_j-14-8(a+b-2)) sum_k s_a s_b.
//    Products of two slices are exact in FP32 and sums of up to 2^24 / 2^14
//    of them stay exact integers, so mma.sync (bf16 in, FP32 accumulate) over
//    a 32-deep k stage returns every pair sum exactly.  Pairs with the same
//    a + b share a weight; their stage sums are added, still exactly, into one
//    64-bit integer per output with a shift of 8 (S+1-(a+b)) bits;
//  * only pairs with a + b <= S + 1 are formed (S (S+1) / 2 products); the
//    dropped ones and the remainders are below 2^(e_i+e_j) 2^(-8S+2) k, so
//    S = 5 gives an error below about 2^-38 k of the operand scales.
//
// The result is converted to FP64 once, at the end.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rk {

namespace {

// Exponent e with |v| < 2^e for the magnitude whose IEEE bits are given
// (0 for zero; subnormals take the smallest normal exponent).
__device__ __forceinline__ int oz_exp(unsigned long long bits) {
    if (bits == 0ull) return 0;
    const int ef = (int)((bits >> 52) & 0x7ff);
    return (ef == 0 ? 1 : ef) - 1022;
}

// Row maxima of |x| as IEEE bit patterns (monotone for non-negative doubles),
// combined with atomicMax.  One CTA covers 32 rows x 256 k of one matrix.
__global__ void __launch_bounds__(256)
k_oz_amax(const double* __restrict__ src, int64_t ld, int64_t stride, int trans, int rows,
          int64_t k, const int64_t* __restrict__ kdev, unsigned long long* __restrict__ amax,
          int rows_pad) {
    const int b = blockIdx.z;
    const double* s = src + (int64_t)b * stride;
    const int64_t kk_n = kdev ? min(k, *kdev) : k;
    const int r0 = blockIdx.y * 32;
    const int64_t k0 = (int64_t)blockIdx.x * 256;
    __shared__ unsigned long long red[32][9];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    unsigned long long m = 0;
    if (trans) {
        // memory runs along rows: lanes over rows, warps over k
        const int r = r0 + tx;
        if (r < rows)
            for (int64_t kk = k0 + ty; kk < min(k0 + 256, kk_n); kk += 8)
                m = max(m, (unsigned long long)__double_as_longlong(fabs(s[kk * ld + r])));
        red[tx][ty] = m;
    } else {
        // memory runs along k: lanes over k, warps over rows (4 each)
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + ty * 4 + q;
            unsigned long long mq = 0;
            if (r < rows)
                for (int64_t kk = k0 + tx; kk < min(k0 + 256, kk_n); kk += 32)
                    mq = max(mq, (unsigned long long)__double_as_longlong(fabs(s[(int64_t)r * ld + kk])));
            for (int o = 16; o > 0; o >>= 1) mq = max(mq, __shfl_xor_sync(0xffffffffu, mq, o));
            if (tx == 0) red[ty * 4 + q][0] = mq;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int r = r0 + threadIdx.x;
        unsigned long long v = red[threadIdx.x][0];
        if (trans)
            for (int q = 1; q < 8; ++q) v = max(v, red[threadIdx.x][q]);
        if (r < rows && v) atomicMax(amax + (int64_t)b * rows_pad + r, v);
    }
}

// Slices of one element, in integer arithmetic (the FP64 pipes are slow):
// F = round(x 2^(7 - e + 8 (S-1))) from the IEEE fields (|F| < 2^(7+8(S-1))),
// then balanced base-256 digits from the bottom: d = ((F + 128) mod 256) - 128,
// F = (F - d) / 256; the last quotient is the top slice (|s_1| <= 128).
template <int S>
__device__ __forceinline__ void oz_digits(double x, int e, uint16_t* dig) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7ff);
    long long F = 0;
    if (ef != 0) {   // zero and subnormals (far below 2^(e - 7 - 8(S-1))) give 0
        const long long mant = (long long)((bits & 0xfffffffffffffull) | 0x10000000000000ull);
        const int sh = ef - 1075 + 7 - e + 8 * (S - 1);   // F = mant 2^sh
        if (sh >= 0)
            F = mant << sh;
        else if (sh > -64)
            F = (mant + (1ll << (-sh - 1))) >> (-sh);
        if (bits >> 63) F = -F;
    }
#pragma unroll
    for (int p = S - 1; p > 0; --p) {
        const long long d = ((F + 128) & 255) - 128;
        dig[p] = (uint16_t)(__float_as_uint((float)d) >> 16);
        F = (F - d) >> 8;
    }
    dig[0] = (uint16_t)(__float_as_uint((float)F) >> 16);
}

// Slices: out[b][q][r][kk] (bf16 bits), rows_pad x kpad per slice, zero in
// the padding.  One CTA covers 32 rows x 64 k; transposed sources go through
// shared memory so that both the reads and the writes are coalesced, and
// each thread stores 8 consecutive k of a row (16 bytes per slice).
template <int S>
__global__ void __launch_bounds__(256)
k_oz_slice(const double* __restrict__ src, int64_t ld, int64_t stride, int trans, int rows,
           int64_t k, const int64_t* __restrict__ kdev,
           const unsigned long long* __restrict__ amax, int rows_pad, int64_t kpad,
           uint16_t* __restrict__ out) {
    const int b = blockIdx.z;
    const double* s = src + (int64_t)b * stride;
    const int64_t kk_n = kdev ? min(k, *kdev) : k;
    const int r0 = blockIdx.y * 32;
    const int64_t k0 = (int64_t)blockIdx.x * 64;
    __shared__ double tile[32][65];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (trans) {
        // lanes along rows: element (row r0 + tx, k k0 + q)
        const int r = r0 + tx;
        for (int q = ty; q < 64; q += 8) {
            const int64_t kk = k0 + q;
            tile[tx][q] = (r < rows && kk < kk_n) ? s[kk * ld + r] : 0.0;
        }
    } else {
        for (int q = ty; q < 32; q += 8) {
            const int r = r0 + q;
            for (int h = 0; h < 2; ++h) {
                const int64_t kk = k0 + tx + 32 * h;
                tile[q][tx + 32 * h] = (r < rows && kk < kk_n) ? s[(int64_t)r * ld + kk] : 0.0;
            }
        }
    }
    __syncthreads();
    const int64_t slice = (int64_t)rows_pad * kpad;
    const int row = threadIdx.x >> 3, c8 = (threadIdx.x & 7) * 8;
    const int r = r0 + row;
    const int64_t kk = k0 + c8;
    if (kk >= kpad) return;
    const int e = r < rows ? oz_exp(amax[(int64_t)b * rows_pad + r]) : 0;
    uint16_t dg[8][S];
#pragma unroll
    for (int q = 0; q < 8; ++q) oz_digits<S>(tile[row][c8 + q], e, dg[q]);
    uint16_t* o = out + (int64_t)b * S * slice + (int64_t)r * kpad + kk;
#pragma unroll
    for (int p = 0; p < S; ++p) {
        uint4 v;
        v.x = dg[0][p] | ((uint32_t)dg[1][p] << 16);
        v.y = dg[2][p] | ((uint32_t)dg[3][p] << 16);
        v.z = dg[4][p] | ((uint32_t)dg[5][p] << 16);
        v.w = dg[6][p] | ((uint32_t)dg[7][p] << 16);
        *reinterpret_cast<uint4*>(o + p * slice) = v;
    }
}

// ---------------------------------------------------------------------------
// C = alpha A B^T (+ beta C) from the slices of A (m rows) and B (n rows).
// CTA tile 64 x 128, k stages of 32 through a double-buffered cp.async
// pipeline; 8 warps of 32 x 32 outputs, each with a 64-bit integer
// accumulator per output.  Shared rows are 64 bytes; the four 16-byte
// chunks of row r sit at chunk c ^ ((r >> 1) & 3), which spreads every
// eight-row ldmatrix over all banks.
constexpr int OBM = 64, OBN = 128, OBK = 32;

__device__ __forceinline__ void oz_cp16(uint32_t saddr, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}

__device__ __forceinline__ void oz_ldm4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void oz_mma(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t oz_swz(int row, int chunk) {
    return (uint32_t)(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
}

template <int S>
struct OzSmem {
    static constexpr int A_BYTES = OBM * OBK * 2;   // one slice of A per stage
    static constexpr int B_BYTES = OBN * OBK * 2;
    static constexpr int STAGE = S * (A_BYTES + B_BYTES);
    static constexpr int BYTES = 2 * STAGE;
};

template <int S>
__global__ void __launch_bounds__(256)
k_oz_gemm(int m, int n, int64_t kpad, int64_t kc, const uint16_t* __restrict__ As,
          const unsigned long long* __restrict__ amaxA, int rowsA_pad,
          const uint16_t* __restrict__ Bs, const unsigned long long* __restrict__ amaxB,
          int rowsB_pad, double alpha, double beta, double* __restrict__ C, int64_t ldc,
          int64_t strideC, int64_t strideSplit, int nsplit, int sym) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int i0 = bi * OBM, j0 = bj * OBN;
    // symmetric: tiles entirely below the diagonal are mirrored from above
    if (sym && j0 + OBN - 1 < i0) return;
    const int b = blockIdx.z / nsplit, split = blockIdx.z % nsplit;
    const int64_t kb = (int64_t)split * kc;
    const int64_t ke = min(kpad, kb + kc);
    extern __shared__ __align__(128) unsigned char oz_sm[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(oz_sm);
    const int64_t sliceA = (int64_t)rowsA_pad * kpad, sliceB = (int64_t)rowsB_pad * kpad;
    const uint16_t* Ab = As + (int64_t)b * S * sliceA + (int64_t)i0 * kpad;
    const uint16_t* Bb = Bs + (int64_t)b * S * sliceB + (int64_t)j0 * kpad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;

    auto load_stage = [&](int buf, int64_t k0) {
        const uint32_t st = sbase + buf * OzSmem<S>::STAGE;
        constexpr int CA = S * OBM * 4, CB = S * OBN * 4;   // 16-byte chunks
        for (int c = tid; c < CA + CB; c += 256) {
            if (c < CA) {
                const int sl = c / (OBM * 4), rem = c % (OBM * 4), row = rem >> 2, ch = rem & 3;
                oz_cp16(st + sl * OzSmem<S>::A_BYTES + oz_swz(row, ch),
                        Ab + sl * sliceA + (int64_t)row * kpad + k0 + ch * 8);
            } else {
                const int cc = c - CA;
                const int sl = cc / (OBN * 4), rem = cc % (OBN * 4), row = rem >> 2, ch = rem & 3;
                oz_cp16(st + S * OzSmem<S>::A_BYTES + sl * OzSmem<S>::B_BYTES + oz_swz(row, ch),
                        Bb + sl * sliceB + (int64_t)row * kpad + k0 + ch * 8);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    long long acc[2][4][4];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
            for (int z = 0; z < 4; ++z) acc[x][y][z] = 0;

    const int nst = (int)((ke - kb + OBK - 1) / OBK);
    if (nst > 0) load_stage(0, kb);
    for (int it = 0; it < nst; ++it) {
        const int buf = it & 1;
        if (it + 1 < nst) {
            load_stage(buf ^ 1, kb + (int64_t)(it + 1) * OBK);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        const uint32_t sa = sbase + buf * OzSmem<S>::STAGE;
        const uint32_t sb = sa + S * OzSmem<S>::A_BYTES;
        // weight classes t = a + b in turn; class t's products go to one of two
        // FP32 accumulator sets while the previous class's sums are folded,
        // so the fold never waits for the tensor pipe to drain
        auto class_mma = [&](int t, float (&f)[2][4][4]) {
#pragma unroll
            for (int x = 0; x < 2; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int z = 0; z < 4; ++z) f[x][y][z] = 0.f;
#pragma unroll 1
            for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                for (int a = 1; a < t; ++a) {
                    const int bsl = t - a;
                    if (a > S || bsl > S) continue;
                    uint32_t af[2][4], bfr[2][4];
                    const int li = lane >> 3, lr = lane & 7;
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi) {
                        const int row = wm * 32 + mi * 16 + lr + 8 * (li & 1);
                        oz_ldm4(sa + (a - 1) * OzSmem<S>::A_BYTES + oz_swz(row, kk * 2 + (li >> 1)),
                                af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
                    }
#pragma unroll
                    for (int np = 0; np < 2; ++np) {
                        const int row = wn * 32 + np * 16 + lr + 8 * (li >> 1);
                        oz_ldm4(sb + (bsl - 1) * OzSmem<S>::B_BYTES + oz_swz(row, kk * 2 + (li & 1)),
                                bfr[np][0], bfr[np][1], bfr[np][2], bfr[np][3]);
                    }
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                        for (int nj = 0; nj < 4; ++nj)
                            oz_mma(f[mi][nj], af[mi], bfr[nj >> 1][(nj & 1) * 2],
                                   bfr[nj >> 1][(nj & 1) * 2 + 1]);
                }
            }
        };
        // fold the exact stage sums of class t (weight 2^(8 (S + 1 - t)))
        auto fold = [&](int t, const float (&f)[2][4][4]) {
            const long long w = 1ll << (8 * (S + 1 - t));
#pragma unroll
            for (int x = 0; x < 2; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int z = 0; z < 4; ++z)
                        acc[x][y][z] += (long long)__float2int_rn(f[x][y][z]) * w;
        };
        float fA[2][4][4], fB[2][4][4];
        class_mma(2, fA);
#pragma unroll
        for (int t = 3; t <= S + 1; ++t) {
            if (t & 1) { class_mma(t, fB); fold(t - 1, fA); }
            else { class_mma(t, fA); fold(t - 1, fB); }
        }
        if ((S + 1) & 1) fold(S + 1, fB);
        else fold(S + 1, fA);
        __syncthreads();
    }

    // epilogue: C_ij = alpha 2^(e_i + e_j - 14 - 8 (S - 1)) acc (+ beta C_ij)
    double* Cb = C + (int64_t)b * strideC + (int64_t)split * strideSplit;
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int hz = 0; hz < 2; ++hz) {
            const int i = i0 + wm * 32 + mi * 16 + g + 8 * hz;
            if (i >= m) continue;
            const int ei = oz_exp(amaxA[(int64_t)b * rowsA_pad + i]);
#pragma unroll
            for (int nj = 0; nj < 4; ++nj)
#pragma unroll
                for (int lz = 0; lz < 2; ++lz) {
                    const int j = j0 + wn * 32 + nj * 8 + 2 * tq + lz;
                    if (j >= n || (sym && j < i)) continue;
                    const int ej = oz_exp(amaxB[(int64_t)b * rowsB_pad + j]);
                    double v = alpha * ldexp((double)acc[mi][nj][hz * 2 + lz], ei + ej - 14 - 8 * (S - 1));
                    double* cp = Cb + (int64_t)i * ldc + j;
                    if (beta != 0.0) v += beta * *cp;
                    *cp = v;
                    if (sym && j != i) Cb[(int64_t)j * ldc + i] = v;
                }
        }
}

template <int S>
cudaError_t oz_gemm_t(int nb, int m, int n, int64_t kpad, int nsplit, const OzOperand& A,
                      const OzOperand& B, double alpha, double beta, double* C, int64_t ldc,
                      int64_t strideC, int64_t strideSplit, int sym, cudaStream_t s) {
    constexpr int smem = OzSmem<S>::BYTES;
    RK_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int64_t kc = round_up(ceil_div(kpad, nsplit), OBK);
    dim3 grid((unsigned)ceil_div(n, OBN), (unsigned)ceil_div(m, OBM), (unsigned)(nb * nsplit));
    k_oz_gemm<S><<<grid, 256, smem, s>>>(m, n, kpad, kc, A.slices, A.amax, A.rows_pad, B.slices,
                                         B.amax, B.rows_pad, alpha, beta, C, ldc, strideC,
                                         strideSplit, nsplit, sym);
    return cudaGetLastError();
}
}  // namespace

int64_t oz_operand_elems(int nb, int S, int rows, int64_t k) {
    return (int64_t)nb * S * round_up(rows, OZ_ROW_PAD) * round_up(k, OZ_K_PAD);
}

cudaError_t launch_oz_split(int nb, int rows, int64_t k, const double* src, int64_t ld,
                            int64_t stride, int trans, const int64_t* kdev, int S, OzOperand& op,
                            cudaStream_t s) {
    if (S != 3 && S != 5) return cudaErrorInvalidValue;
    op.S = S;
    op.rows = rows;
    op.rows_pad = (int)round_up(rows, OZ_ROW_PAD);
    op.kpad = round_up(k, OZ_K_PAD);
    if (nb <= 0 || rows <= 0 || k <= 0) return cudaSuccess;
    RK_CUDA_TRY(cudaMemsetAsync(op.amax, 0, sizeof(unsigned long long) * nb * op.rows_pad, s));
    dim3 ga((unsigned)ceil_div(k, 256), (unsigned)ceil_div(rows, 32), (unsigned)nb);
    k_oz_amax<<<ga, 256, 0, s>>>(src, ld, stride, trans, rows, k, kdev, op.amax, op.rows_pad);
    RK_CUDA_TRY(cudaGetLastError());
    dim3 gs((unsigned)ceil_div(op.kpad, 64), (unsigned)(op.rows_pad / 32), (unsigned)nb);
    if (S == 3)
        k_oz_slice<3><<<gs, 256, 0, s>>>(src, ld, stride, trans, rows, k, kdev, op.amax,
                                         op.rows_pad, op.kpad, op.slices);
    else
        k_oz_slice<5><<<gs, 256, 0, s>>>(src, ld, stride, trans, rows, k, kdev, op.amax,
                                         op.rows_pad, op.kpad, op.slices);
    return cudaGetLastError();
}

cudaError_t launch_oz_gemm(int nb, int m, int n, const OzOperand& A, const OzOperand& B,
                           double alpha, double beta, double* C, int64_t ldc, int64_t strideC,
                           int sym, cudaStream_t s, int nsplit, int64_t strideSplit) {
    if (A.S != B.S || A.kpad != B.kpad || m > A.rows_pad || n > B.rows_pad || nsplit < 1)
        return cudaErrorInvalidValue;
    if (sym && m != n) return cudaErrorInvalidValue;
    if (nb <= 0 || m <= 0 || n <= 0) return cudaSuccess;
    if (A.tc)
        return launch_oz_gemm_tc(nb, m, n, A, B, alpha, beta, C, ldc, strideC, sym, s, nsplit,
                                 strideSplit, A.err);
    if (A.S == 3)
        return oz_gemm_t<3>(nb, m, n, A.kpad, nsplit, A, B, alpha, beta, C, ldc, strideC,
                            strideSplit, sym, s);
    return oz_gemm_t<5>(nb, m, n, A.kpad, nsplit, A, B, alpha, beta, C, ldc, strideC, strideSplit,
                        sym, s);
}

}  // namespace rk
