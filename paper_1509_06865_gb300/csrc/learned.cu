// The learned smoother: a three-layer 4D convolutional network that stands in
// for the SAP smoother M of the two-grid cycle (Eq. 2.3) inside the flexible
// outer FGMRES (Sec. 2.2), trained on the GPU on (residual, SAP correction)
// pairs that the method itself produces.  The paper has no learned smoother; a
// poor network changes the outer iteration count, never the solution.
//
// Network (every layer a 3^4 convolution on the periodic lattice, no bias):
//   x = r / ||r||  as 24 real channels (2k = Re r_k, 2k+1 = Im r_k, k = 3 spin + colour)
//   f(x) = W3 * gelu(W2 * gelu(W1 * x)),  24 -> 32 -> 32 -> 24 channels
//   M(r) = ||r|| f(r / ||r||)
// gelu in its tanh form (Hendrycks and Gimpel 2016).  Loss of a batch of N pairs
// L = 1/(2N) sum ||f(x_n) - t_n||^2 with t_n = SAP(r_n) / ||r_n||; Adam (Kingma
// and Ba 2015) on FP32 master weights.
//
// Data layout: activations BF16 [site][32 channels] (64 bytes a site, channels
// beyond a layer's width zero), pre-activations and outputs FP32 [site][32];
// weights [layer][tap 81][out 32][in 32], master FP32, BF16 copies for the
// forward product and, transposed and reflected, for the data gradient.
// A batch of B fields is B independent periodic lattices, one after another.
//
// Products on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation; operands staged in shared memory and loaded with ldmatrix):
//   forward / data gradient   out(s)[o] = sum_tap sum_i W[tap][o][i] in(s + tap)[i]
//                             M = sites, N = out, K = (tap, in); a CTA owns a
//                             4 x 4 x 4 x 2 box of sites and stages it with its
//                             one-site halo, and the weights nine taps at a time
//   weight gradient           dW[tap][o][i] = sum_s dz(s)[o] in(s + tap)[i]
//                             M = out, N = in, K = sites (ldmatrix.trans), one
//                             tap and a chunk of boxes per CTA, FP32 atomics
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>

#include "internal.h"

namespace mgeig {

namespace {

constexpr int NC = 32;                 // padded channel count
constexpr int NTAPS = 81;
constexpr int BX = 4, BY = 4, BZ = 4, BT = 2;   // site box of a CTA
constexpr int BOX = BX * BY * BZ * BT;          // 128 sites, 4 warps x 32
constexpr int HX = BX + 2, HY = BY + 2, HZ = BZ + 2, HT = BT + 2;
constexpr int HALO = HX * HY * HZ * HT;         // 864 rows
constexpr int TAPS_PER_STAGE = 9;
constexpr int CONV_THREADS = 128;
constexpr int WG_BOXES = 16;                    // boxes per weight-gradient CTA
constexpr float GELU_C = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float GELU_A = 0.044715f;

struct LatDims {
    int L[4];        // x, y, z, t extents of one field
    int V;           // sites per field
    int nb[4];       // boxes per direction
    int boxes;       // boxes per field
};

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.f + tanhf(GELU_C * (z + GELU_A * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float th = tanhf(GELU_C * (z + GELU_A * z * z * z));
    return 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * GELU_C * (1.f + 3.f * GELU_A * z * z);
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const void *smem_row) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t r[4], const void *smem_row) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::);
}

// tap index -> offset; tap = ((dt+1)*3 + (dz+1))*9 + (dy+1)*3 + (dx+1)
__host__ __device__ __forceinline__ void tap_offset(int tap, int d[4]) {
    d[0] = tap % 3 - 1;
    d[1] = (tap / 3) % 3 - 1;
    d[2] = (tap / 9) % 3 - 1;
    d[3] = tap / 27 - 1;
}

// first site (field, box) of CTA box index b; coordinates of local site l
__device__ __forceinline__ void box_origin(const LatDims &D, int b, int &field, int o[4]) {
    field = b / D.boxes;
    int r = b % D.boxes;
    o[0] = (r % D.nb[0]) * BX; r /= D.nb[0];
    o[1] = (r % D.nb[1]) * BY; r /= D.nb[1];
    o[2] = (r % D.nb[2]) * BZ;
    o[3] = (r / D.nb[2]) * BT;
}
__device__ __forceinline__ void local_coords(int l, int c[4]) {
    c[0] = l % BX; l /= BX;
    c[1] = l % BY; l /= BY;
    c[2] = l % BZ;
    c[3] = l / BZ;
}
__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }
__device__ __forceinline__ size_t site_index(const LatDims &D, int field, const int x[4]) {
    return (size_t)field * D.V + (((size_t)x[3] * D.L[2] + x[2]) * D.L[1] + x[1]) * D.L[0] + x[0];
}

enum Epi { EPI_GELU = 0, EPI_OUT = 1, EPI_DGELU = 2 };

struct ConvArgs {
    LatDims D;
    const __nv_bfloat16 *in;     // [B V][32]
    const __nv_bfloat16 *W;      // [81][32 out][32 in]
    float *z;                    // EPI_GELU: pre-activation out; EPI_OUT: output
    __nv_bfloat16 *act;          // EPI_GELU: gelu(z); EPI_DGELU: gradient times gelu'(zprev)
    const float *zprev;          // EPI_DGELU: pre-activation of the layer below
    int cout;                    // output channels that are kept (the rest written as zero)
};

// Staged rows of 32 BF16 channels are 64 bytes, four 16-byte chunks.  An 8-row
// ldmatrix phase over consecutive rows would hit each bank four times, so chunk c
// of row r is stored at chunk c ^ ((r >> 1) & 3): rows 2k and 2k + 1 share a
// pattern, four row pairs cover the 32 banks.
__device__ __forceinline__ int swz(int row, int chunk) { return row * NC + 8 * (chunk ^ ((row >> 1) & 3)); }

// out(s)[o] = sum_tap sum_i W[tap][o][i] in(s + tap)[i] for one box of sites
template <int EPI>
__global__ void __launch_bounds__(CONV_THREADS) conv_kernel(ConvArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16 *halo = reinterpret_cast<__nv_bfloat16 *>(smem);              // [HALO][32]
    __nv_bfloat16 *wst = halo + (size_t)HALO * NC;                              // [9][32][32]
    static_assert(HALO % 32 == 0, "the halo rows come in groups of 32");
    int field, o[4];
    box_origin(a.D, blockIdx.x, field, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the box and its halo, 16-byte async copies, periodic wrap: warp w takes the
    // groups of 32 rows w, w + 4, ...; each lane works out the global offset of
    // one row of the group, then four lanes at a time copy a row's four chunks
    // (64 contiguous bytes) with the offset taken from the lane that owns it
    for (int r0 = 32 * w; r0 < HALO; r0 += CONV_THREADS) {
        int h = r0 + lane;
        int x[4];
        x[0] = wrap(o[0] + h % HX - 1, a.D.L[0]); h /= HX;
        x[1] = wrap(o[1] + h % HY - 1, a.D.L[1]); h /= HY;
        x[2] = wrap(o[2] + h % HZ - 1, a.D.L[2]);
        x[3] = wrap(o[3] + h / HZ - 1, a.D.L[3]);
        const long long off = (long long)site_index(a.D, field, x) * NC;
        const int ch = lane & 3;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int src = 8 * k + (lane >> 2);
            const long long o_src = __shfl_sync(0xffffffffu, off, src);
            cp_async16(halo + swz(r0 + src, ch), a.in + o_src + ch * 8);
        }
    }
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) acc[mi][nj][0] = acc[mi][nj][1] = acc[mi][nj][2] = acc[mi][nj][3] = 0.f;
    // the lane's A rows: site 32 w + 16 mi + (lane % 8) + 8 ((lane / 8) % 2), channel offset 8 (lane / 16)
    int lc[2][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) local_coords(32 * w + 16 * mi + (lane & 7) + 8 * ((lane >> 3) & 1), lc[mi]);
    const int a_ch = 8 * (lane >> 4);
    // the lane's B rows: out channel 8 (pair) + (lane % 8) + 8 (lane / 16), in offset 8 ((lane / 8) % 2)
    const int b_row = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
    for (int t0 = 0; t0 < NTAPS; t0 += TAPS_PER_STAGE) {
        __syncthreads();   // the previous weights are no longer read
        for (int e = threadIdx.x; e < TAPS_PER_STAGE * NC * NC / 8; e += blockDim.x)
            cp_async16(wst + swz(e >> 2, e & 3), a.W + (size_t)t0 * NC * NC + (size_t)e * 8);
        cp_async_wait_all();
        __syncthreads();
        for (int tt = 0; tt < TAPS_PER_STAGE; ++tt) {
            int d[4];
            tap_offset(t0 + tt, d);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t af[2][4];
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    const int h = (((lc[mi][3] + 1 + d[3]) * HZ + (lc[mi][2] + 1 + d[2])) * HY +
                                   (lc[mi][1] + 1 + d[1])) * HX + (lc[mi][0] + 1 + d[0]);
                    ldmatrix_x4(af[mi], halo + swz(h, 2 * ks + (a_ch >> 3)));
                }
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    uint32_t bf[4];
                    ldmatrix_x4(bf, wst + swz(tt * NC + 16 * np + b_row, 2 * ks + (b_k >> 3)));
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi) {
                        mma16816(acc[mi][2 * np], af[mi], bf[0], bf[1]);
                        mma16816(acc[mi][2 * np + 1], af[mi], bf[2], bf[3]);
                    }
                }
            }
        }
    }
    // epilogue: fragment element e of (mi, nj) is row g + 8 (e / 2), column 8 nj + 2 (lane % 4) + e % 2
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            int c[4], x[4];
            local_coords(32 * w + 16 * mi + g + 8 * half, c);
            for (int k = 0; k < 4; ++k) x[k] = o[k] + c[k];
            const size_t s = site_index(a.D, field, x);
#pragma unroll
            for (int nj = 0; nj < 4; ++nj) {
                const int col = 8 * nj + 2 * tq;
                float v0 = acc[mi][nj][2 * half], v1 = acc[mi][nj][2 * half + 1];
                if (col >= a.cout) v0 = 0.f;
                if (col + 1 >= a.cout) v1 = 0.f;
                if (EPI == EPI_GELU) {
                    *reinterpret_cast<float2 *>(a.z + s * NC + col) = make_float2(v0, v1);
                    *reinterpret_cast<__nv_bfloat162 *>(a.act + s * NC + col) =
                        __floats2bfloat162_rn(col < a.cout ? gelu(v0) : 0.f, col + 1 < a.cout ? gelu(v1) : 0.f);
                } else if (EPI == EPI_OUT) {
                    *reinterpret_cast<float2 *>(a.z + s * NC + col) = make_float2(v0, v1);
                } else {
                    const float2 zp = *reinterpret_cast<const float2 *>(a.zprev + s * NC + col);
                    *reinterpret_cast<__nv_bfloat162 *>(a.act + s * NC + col) =
                        __floats2bfloat162_rn(v0 * gelu_grad(zp.x), v1 * gelu_grad(zp.y));
                }
            }
        }
}

// dW[tap][o][i] += sum_s dz(s)[o] in(s + tap)[i] over WG_BOXES boxes of sites
__global__ void __launch_bounds__(CONV_THREADS) wgrad_kernel(LatDims D, int nboxes, const __nv_bfloat16 *in,
                                                             const __nv_bfloat16 *dz, float *dW) {
    static_assert(BOX == CONV_THREADS, "one staged site per thread");
    __shared__ __align__(16) __nv_bfloat16 xs[BOX * NC];   // in(s + tap) of the box's sites (swizzled rows)
    __shared__ __align__(16) __nv_bfloat16 gs[BOX * NC];   // dz(s) (swizzled rows)
    __shared__ float red[4][NC * NC / 4];                  // warp partials, 1/4 at a time
    const int tap = blockIdx.y;
    int d[4];
    tap_offset(tap, d);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float acc[2][4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) acc[mi][nj][0] = acc[mi][nj][1] = acc[mi][nj][2] = acc[mi][nj][3] = 0.f;
    for (int bb = 0; bb < WG_BOXES; ++bb) {
        const int b = blockIdx.x * WG_BOXES + bb;
        if (b >= nboxes) break;   // the same for the whole CTA
        int field, o[4];
        box_origin(D, b, field, o);
        __syncthreads();
        // warp w stages sites 32 w .. 32 w + 31: each lane works out the offsets
        // of one site, then four lanes at a time copy a site's four chunks
        // (64 contiguous bytes) with the offsets taken from the lane that owns it
        {
            int c[4], x[4], y[4];
            local_coords(32 * w + lane, c);
            for (int k = 0; k < 4; ++k) { x[k] = o[k] + c[k]; y[k] = wrap(x[k] + d[k], D.L[k]); }
            const long long og = (long long)site_index(D, field, x) * NC;
            const long long ox = (long long)site_index(D, field, y) * NC;
            const int ch = lane & 3;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int src = 8 * k + (lane >> 2);
                const long long g_off = __shfl_sync(0xffffffffu, og, src);
                const long long x_off = __shfl_sync(0xffffffffu, ox, src);
                cp_async16(gs + swz(32 * w + src, ch), dz + g_off + ch * 8);
                cp_async16(xs + swz(32 * w + src, ch), in + x_off + ch * 8);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // warp w: sites 32 w .. 32 w + 31, two k steps of 16 sites
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int s0 = 32 * w + 16 * ks;
            uint32_t af[2][4];
            // A (out x sites) from dz rows (sites x out), transposed: matrix j = (out 8 (j % 2), sites 8 (j / 2))
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldmatrix_x4_trans(af[mi], gs + swz(s0 + (lane & 7) + 8 * (lane >> 4), 2 * mi + ((lane >> 3) & 1)));
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t bf[4];
                // B (sites x in) from the rows of in(s + tap): matrix j = (sites 8 (j % 2), in 8 (2 np + j / 2))
                ldmatrix_x4_trans(bf, xs + swz(s0 + (lane & 7) + 8 * ((lane >> 3) & 1), 2 * np + (lane >> 4)));
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma16816(acc[mi][2 * np], af[mi], bf[0], bf[1]);
                    mma16816(acc[mi][2 * np + 1], af[mi], bf[2], bf[3]);
                }
            }
        }
    }
    // reduce the four warps' 32 x 32 partials, one quarter (8 rows of out) at a time
    const int g = lane >> 2, tq = lane & 3;
    for (int q = 0; q < 4; ++q) {
        __syncthreads();
        const int mi = q >> 1, half = q & 1;   // rows 16 mi + 8 half + g
#pragma unroll
        for (int nj = 0; nj < 4; ++nj) {
            red[w][g * NC + 8 * nj + 2 * tq] = acc[mi][nj][2 * half];
            red[w][g * NC + 8 * nj + 2 * tq + 1] = acc[mi][nj][2 * half + 1];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 8 * NC; e += blockDim.x) {
            const float v = red[0][e] + red[1][e] + red[2][e] + red[3][e];
            const int row = 16 * mi + 8 * half + e / NC, col = e % NC;
            atomicAdd(dW + ((size_t)tap * NC + row) * NC + col, v);
        }
    }
}

// level-precision spinors (FP32 [6][V] float4) -> BF16 channels [site][32] times s
__global__ void spinor_to_channels_kernel(int V, int nfield, const float4 *psi, size_t fstride, const float *scale,
                                          __nv_bfloat16 *x) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * nfield) return;
    const int f = (int)(i / V), s = (int)(i % V);
    const float sc = scale[f];
    const float4 *p = psi + f * fstride;
    __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(x + i * NC);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = p[(size_t)q * V + s];
        o[2 * q] = __floats2bfloat162_rn(sc * v.x, sc * v.y);
        o[2 * q + 1] = __floats2bfloat162_rn(sc * v.z, sc * v.w);
    }
#pragma unroll
    for (int q = 12; q < 16; ++q) o[q] = __floats2bfloat162_rn(0.f, 0.f);
}

// FP32 spinors -> FP32 channels [site][32] times s (training targets)
__global__ void spinor_to_channels_f32_kernel(int V, int nfield, const float4 *psi, size_t fstride,
                                              const float *scale, float *t) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * nfield) return;
    const int f = (int)(i / V), s = (int)(i % V);
    const float sc = scale[f];
    const float4 *p = psi + f * fstride;
    float4 *o = reinterpret_cast<float4 *>(t + i * NC);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = p[(size_t)q * V + s];
        o[q] = make_float4(sc * v.x, sc * v.y, sc * v.z, sc * v.w);
    }
#pragma unroll
    for (int q = 6; q < 8; ++q) o[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// z += s * channels(y): FP32 channels [site][32] back into one FP32 spinor
__global__ void channels_add_to_spinor_kernel(int V, const float *y, const float *scale, float4 *z) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const float sc = scale[0];
    const float4 *yi = reinterpret_cast<const float4 *>(y + (size_t)s * NC);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = yi[q];
        float4 zz = z[(size_t)q * V + s];
        zz.x += sc * v.x; zz.y += sc * v.y; zz.z += sc * v.z; zz.w += sc * v.w;
        z[(size_t)q * V + s] = zz;
    }
}

// scale[f] = 1 / sqrt(norm2[f]) (0 for a zero field), from the reduction results
__global__ void inv_norm_kernel(int n, const double2 *norm2, float *inv, float *nrm) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const double v = norm2[f].x;
    inv[f] = v > 0 ? (float)(1.0 / sqrt(v)) : 0.f;
    if (nrm) nrm[f] = (float)sqrt(v > 0 ? v : 0.0);
}

// d = y - t; loss partial sums (per block, FP64); dy = d / N in BF16
__global__ void loss_grad_kernel(size_t n, const float *y, const float *t, float invN, __nv_bfloat16 *dy,
                                 double *partial) {
    double acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        dy[i] = __float2bfloat16_rn(d * invN);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

// Adam on the FP32 master weights; refreshes the BF16 forward copy Wf[l][tap][o][i]
// and the data-gradient copy Wt[l][tap'][i][o] = Wf[l][80 - tap'][o][i] (reflected tap)
__global__ void adam_kernel(int n, float *W, const float *G, float *m, float *v, float lr, float b1, float b2,
                            float c1, float c2, float eps, __nv_bfloat16 *Wf, __nv_bfloat16 *Wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float w = W[e];
    if (G) {
        const float gg = G[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        w -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        W[e] = w;
    }
    const int i = e % NC, o = (e / NC) % NC, tap = (e / (NC * NC)) % NTAPS, l = e / (NC * NC * NTAPS);
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    Wf[e] = b;
    Wt[(((size_t)l * NTAPS + (NTAPS - 1 - tap)) * NC + i) * NC + o] = b;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

struct Net {
    int cin[3] = {24, 32, 32}, cout[3] = {32, 32, 24};
    DevBuf W, G, m, v, Wf, Wt;          // [3][81][32][32]
    int step = 0;
    bool ready = false;
    // activations of a batch
    int batch = 0;
    DevBuf x, a1, a2, dz, z1, z2, y, t, dyb;
    DevBuf lossp, scal;                 // loss partial sums; per-field scales
};

static size_t wcount() { return (size_t)3 * NTAPS * NC * NC; }

static LatDims lat(const Ctx &c) {
    LatDims D;
    for (int mu = 0; mu < 4; ++mu) D.L[mu] = c.dims[mu];
    D.V = c.g.V;
    D.nb[0] = c.dims[0] / BX; D.nb[1] = c.dims[1] / BY; D.nb[2] = c.dims[2] / BZ; D.nb[3] = c.dims[3] / BT;
    D.boxes = D.nb[0] * D.nb[1] * D.nb[2] * D.nb[3];
    return D;
}

bool net_supported_dims(const int dims[4]) {
    return dims[0] % BX == 0 && dims[1] % BY == 0 && dims[2] % BZ == 0 && dims[3] % BT == 0;
}
bool net_supported(const Ctx &c) { return net_supported_dims(c.dims); }

static Net &net(Ctx &c) {
    MG_REQUIRE(net_supported(c), MGEIG_EINVAL);
    if (!c.net) c.net = new Net();
    Net &n = *c.net;
    if (!n.W.p) {
        const size_t nw = wcount();
        n.W.alloc(nw * 4); n.G.alloc(nw * 4); n.m.alloc(nw * 4); n.v.alloc(nw * 4);
        n.Wf.alloc(nw * 2); n.Wt.alloc(nw * 2);
        MG_CUDA(cudaMemsetAsync(n.W.p, 0, nw * 4, c.stream));
        MG_CUDA(cudaMemsetAsync(n.m.p, 0, nw * 4, c.stream));
        MG_CUDA(cudaMemsetAsync(n.v.p, 0, nw * 4, c.stream));
        n.lossp.alloc(1024 * sizeof(double));
        n.scal.alloc(2 * 64 * sizeof(float));
    }
    return n;
}

static void net_batch(Ctx &c, Net &n, int batch) {
    if (n.batch >= batch) return;
    const size_t sites = (size_t)c.g.V * batch;
    n.x.alloc(sites * NC * 2); n.a1.alloc(sites * NC * 2); n.a2.alloc(sites * NC * 2); n.dz.alloc(sites * NC * 2);
    n.dyb.alloc(sites * NC * 2);
    n.z1.alloc(sites * NC * 4); n.z2.alloc(sites * NC * 4); n.y.alloc(sites * NC * 4); n.t.alloc(sites * NC * 4);
    n.batch = batch;
}

void net_free(Ctx &c) {
    if (!c.net) return;
    Net &n = *c.net;
    for (DevBuf *b : {&n.W, &n.G, &n.m, &n.v, &n.Wf, &n.Wt, &n.x, &n.a1, &n.a2, &n.dz, &n.z1, &n.z2, &n.y, &n.t,
                      &n.dyb, &n.lossp, &n.scal})
        b->free();
    delete c.net;
    c.net = nullptr;
}

// refreshes the BF16 copies from the master weights (no update)
static void refresh(Ctx &c, Net &n) {
    const int nw = (int)wcount();
    adam_kernel<<<grid_for(nw, 256), 256, 0, c.stream>>>(nw, n.W.as<float>(), nullptr, nullptr, nullptr, 0, 0, 0, 1,
                                                         1, 0, n.Wf.as<__nv_bfloat16>(), n.Wt.as<__nv_bfloat16>());
    MG_CHECK_LAUNCH();
    n.ready = true;
}

void net_set_weights(Ctx &c, const float *host) {
    Net &n = net(c);
    MG_CUDA(cudaMemcpyAsync(n.W.p, host, wcount() * 4, cudaMemcpyHostToDevice, c.stream));
    MG_CUDA(cudaMemsetAsync(n.m.p, 0, wcount() * 4, c.stream));
    MG_CUDA(cudaMemsetAsync(n.v.p, 0, wcount() * 4, c.stream));
    n.step = 0;
    refresh(c, n);
    sync(c);
}

void net_get_weights(Ctx &c, float *host) {
    Net &n = net(c);
    MG_CUDA(cudaMemcpyAsync(host, n.W.p, wcount() * 4, cudaMemcpyDeviceToHost, c.stream));
    sync(c);
}

// He-normal initialisation (std 0.5 sqrt(2 / fan_in), fan_in = 81 c_in) from a
// 64-bit Mersenne twister and Box-Muller: the same weights on every host
void net_init(Ctx &c, uint64_t seed) {
    std::vector<float> W(wcount(), 0.f);
    std::mt19937_64 rng(seed);
    auto uni = [&]() { return ((rng() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    const int cin[3] = {24, 32, 32}, cout[3] = {32, 32, 24};
    for (int l = 0; l < 3; ++l) {
        const double sd = 0.5 * std::sqrt(2.0 / (NTAPS * cin[l]));
        for (int tap = 0; tap < NTAPS; ++tap)
            for (int o = 0; o < cout[l]; ++o)
                for (int i = 0; i < cin[l]; ++i) {
                    const double u1 = uni(), u2 = uni();
                    const double gauss = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
                    W[(((size_t)l * NTAPS + tap) * NC + o) * NC + i] = (float)(sd * gauss);
                }
    }
    net_set_weights(c, W.data());
}

static size_t conv_smem() { return (size_t)HALO * NC * 2 + (size_t)TAPS_PER_STAGE * NC * NC * 2; }

template <int EPI>
static void launch_conv(Ctx &c, int batch, const void *in, const void *W, float *z, void *act, const float *zprev,
                        int cout) {
    ConvArgs a;
    a.D = lat(c);
    a.in = static_cast<const __nv_bfloat16 *>(in);
    a.W = static_cast<const __nv_bfloat16 *>(W);
    a.z = z;
    a.act = static_cast<__nv_bfloat16 *>(act);
    a.zprev = zprev;
    a.cout = cout;
    const size_t smem = conv_smem();
    MG_CUDA(cudaFuncSetAttribute(conv_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TimeScope ts(c.timer, K_NET, (double)batch * c.g.V * (2 * NC * 2 + NC * 4) + NTAPS * NC * NC * 2.0);
    conv_kernel<EPI><<<a.D.boxes * batch, CONV_THREADS, smem, c.stream>>>(a);
    MG_CHECK_LAUNCH();
}

static const __nv_bfloat16 *wf(Net &n, int l) { return n.Wf.as<__nv_bfloat16>() + (size_t)l * NTAPS * NC * NC; }
static const __nv_bfloat16 *wt(Net &n, int l) { return n.Wt.as<__nv_bfloat16>() + (size_t)l * NTAPS * NC * NC; }

// forward pass of a batch whose input channels are in n.x: y in n.y
static void forward(Ctx &c, Net &n, int batch) {
    launch_conv<EPI_GELU>(c, batch, n.x.p, wf(n, 0), n.z1.as<float>(), n.a1.p, nullptr, n.cout[0]);
    launch_conv<EPI_GELU>(c, batch, n.a1.p, wf(n, 1), n.z2.as<float>(), n.a2.p, nullptr, n.cout[1]);
    launch_conv<EPI_OUT>(c, batch, n.a2.p, wf(n, 2), n.y.as<float>(), nullptr, nullptr, n.cout[2]);
}

static void wgrad(Ctx &c, int batch, const void *in, const void *dz, float *dW) {
    const LatDims D = lat(c);
    const int nboxes = D.boxes * batch;
    dim3 grid((nboxes + WG_BOXES - 1) / WG_BOXES, NTAPS);
    TimeScope ts(c.timer, K_NET, (double)nboxes * BOX * NC * 2 * 2 + NTAPS * NC * NC * 4.0);
    wgrad_kernel<<<grid, CONV_THREADS, 0, c.stream>>>(D, nboxes, static_cast<const __nv_bfloat16 *>(in),
                                                      static_cast<const __nv_bfloat16 *>(dz), dW);
    MG_CHECK_LAUNCH();
}

// loss of the batch against n.t and the weight gradients into n.G; returns the
// loss (a device-to-host read)
static double backward(Ctx &c, Net &n, int batch) {
    const size_t ne = (size_t)c.g.V * batch * NC;
    const int nb = std::min<int>(1024, grid_for(ne, 256));
    loss_grad_kernel<<<nb, 256, 0, c.stream>>>(ne, n.y.as<float>(), n.t.as<float>(), 1.f / batch,
                                               n.dyb.as<__nv_bfloat16>(), n.lossp.as<double>());
    MG_CHECK_LAUNCH();
    float *G = n.G.as<float>();
    const size_t per = (size_t)NTAPS * NC * NC;
    MG_CUDA(cudaMemsetAsync(G, 0, wcount() * 4, c.stream));
    wgrad(c, batch, n.a2.p, n.dyb.p, G + 2 * per);
    launch_conv<EPI_DGELU>(c, batch, n.dyb.p, wt(n, 2), nullptr, n.dz.p, n.z2.as<float>(), n.cin[2]);
    wgrad(c, batch, n.a1.p, n.dz.p, G + per);
    // the data gradient of layer 2 overwrites dz only after its weight gradient read it: reuse dyb
    launch_conv<EPI_DGELU>(c, batch, n.dz.p, wt(n, 1), nullptr, n.dyb.p, n.z1.as<float>(), n.cin[1]);
    wgrad(c, batch, n.x.p, n.dyb.p, G);
    std::vector<double> lp(nb);
    MG_CUDA(cudaMemcpyAsync(lp.data(), n.lossp.p, nb * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    double L = 0;
    for (double v : lp) L += v;
    return 0.5 * L / batch;
}

static void adam(Ctx &c, Net &n, double lr) {
    n.step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n.step), c2 = 1.f - std::pow(b2, (float)n.step);
    const int nw = (int)wcount();
    adam_kernel<<<grid_for(nw, 256), 256, 0, c.stream>>>(nw, n.W.as<float>(), n.G.as<float>(), n.m.as<float>(),
                                                         n.v.as<float>(), (float)lr, b1, b2, c1, c2, 1e-8f,
                                                         n.Wf.as<__nv_bfloat16>(), n.Wt.as<__nv_bfloat16>());
    MG_CHECK_LAUNCH();
}

// loss and gradients for host inputs: x, t as FP64 channels [batch][V][24]
double net_loss_grads(Ctx &c, const double *x, const double *t, int batch, float *G_host) {
    Net &n = net(c);
    MG_REQUIRE(n.ready, MGEIG_ENOTSETUP);
    net_batch(c, n, batch);
    const size_t sites = (size_t)c.g.V * batch;
    std::vector<__nv_bfloat16> xb(sites * NC);
    std::vector<float> tf(sites * NC, 0.f);
    for (size_t s = 0; s < sites; ++s)
        for (int k = 0; k < NC; ++k) {
            xb[s * NC + k] = __float2bfloat16_rn(k < 24 ? (float)x[s * 24 + k] : 0.f);
            if (k < 24) tf[s * NC + k] = (float)t[s * 24 + k];
        }
    MG_CUDA(cudaMemcpyAsync(n.x.p, xb.data(), xb.size() * 2, cudaMemcpyHostToDevice, c.stream));
    MG_CUDA(cudaMemcpyAsync(n.t.p, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, c.stream));
    forward(c, n, batch);
    const double L = backward(c, n, batch);
    MG_CUDA(cudaMemcpyAsync(G_host, n.G.p, wcount() * 4, cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    return L;
}

// z += M(r) = ||r|| f(r / ||r||) for one level-precision (FP32) spinor r
void net_smooth(Ctx &c, const void *r, void *z) {
    Net &n = net(c);
    MG_REQUIRE(n.ready, MGEIG_ENOTSETUP);
    net_batch(c, n, 1);
    const size_t N = c.fine_ncpx();
    cpx<double> *nrm = reinterpret_cast<cpx<double> *>(n.lossp.p);
    blas_norm2<float>(c, r, N, nrm);
    float *inv = n.scal.as<float>(), *val = inv + 64;
    inv_norm_kernel<<<1, 32, 0, c.stream>>>(1, reinterpret_cast<const double2 *>(nrm), inv, val);
    MG_CHECK_LAUNCH();
    spinor_to_channels_kernel<<<grid_for(c.g.V, 256), 256, 0, c.stream>>>(
        c.g.V, 1, static_cast<const float4 *>(r), 0, inv, n.x.as<__nv_bfloat16>());
    MG_CHECK_LAUNCH();
    forward(c, n, 1);
    channels_add_to_spinor_kernel<<<grid_for(c.g.V, 256), 256, 0, c.stream>>>(c.g.V, n.y.as<float>(), val,
                                                                               static_cast<float4 *>(z));
    MG_CHECK_LAUNCH();
}

// one training step on `batch` pairs whose inputs r_f (FP32 spinors, back to back)
// and SAP corrections e_f are given: x = r / ||r||, t = e / ||r||
double net_train_step(Ctx &c, const void *r, const void *e, int batch, double lr) {
    Net &n = net(c);
    MG_REQUIRE(n.ready && batch <= 64, MGEIG_EINVAL);
    net_batch(c, n, batch);
    const size_t N = c.fine_ncpx(), fb = N * 8;
    cpx<double> *nrm = reinterpret_cast<cpx<double> *>(n.lossp.p);
    for (int f = 0; f < batch; ++f) blas_norm2<float>(c, static_cast<const char *>(r) + fb * f, N, nrm + f);
    float *inv = n.scal.as<float>();
    inv_norm_kernel<<<1, 64, 0, c.stream>>>(batch, reinterpret_cast<const double2 *>(nrm), inv, nullptr);
    MG_CHECK_LAUNCH();
    const size_t sites = (size_t)c.g.V * batch;
    spinor_to_channels_kernel<<<grid_for(sites, 256), 256, 0, c.stream>>>(
        c.g.V, batch, static_cast<const float4 *>(r), (size_t)6 * c.g.V, inv, n.x.as<__nv_bfloat16>());
    MG_CHECK_LAUNCH();
    spinor_to_channels_f32_kernel<<<grid_for(sites, 256), 256, 0, c.stream>>>(
        c.g.V, batch, static_cast<const float4 *>(e), (size_t)6 * c.g.V, inv, n.t.as<float>());
    MG_CHECK_LAUNCH();
    forward(c, n, batch);
    const double L = backward(c, n, batch);
    adam(c, n, lr);
    return L;
}

}  // namespace mgeig
