// The coarse operator with 16-bit links (the precision split of Sec. 2.2 taken
// one level further: the coarse operator D_c = P^dag D P of Eq. 2.5 stored in
// bfloat16 or IEEE half, one FP32 scale per 2N_tv x 2N_tv link block, every
// product accumulated in FP32).
//
//   compress_coarse        FP32 blocks Dc[d][site][col][row] -> 16-bit planes
//                          L[d][site][re|im][row][col] (entries divided by the
//                          block's largest |re|, |im|) and scale[d][site]
//   coarse_apply_links16   y = (Q_c - sigma) x (or the D_c form), one right-hand
//                          side, thread per coarse row
//   coarse_apply_nrhs      Y = (Q_c - sigma) X for nrhs <= 16 right-hand sides
//                          on the tensor cores (mma.sync m16n8k16, BF16 in, FP32
//                          accumulate): per coarse site
//                              [P | Q] = [Ar ; Ai] (s_d [Xr | Xi]) summed over the
//                          nine hops d, Yr = P_r - Q_i, Yi = P_i + Q_r (complex
//                          product from real 40 x 40 planes), the per-link scale
//                          s_d folded into the staged right-hand sides
#include "half16.cuh"
#include "internal.h"

namespace mgeig {

// ---------------------------------------------------------------------------
// compression: one CTA per (direction, coarse site) block

template <typename H>
__global__ void __launch_bounds__(256) compress_coarse_kernel(int n2, const float2 *__restrict__ Dc, H *__restrict__ L,
                                                              float *__restrict__ scale) {
    const size_t blk = blockIdx.x;
    const float2 *src = Dc + blk * n2 * n2;   // column-major: src[col * n2 + row]
    H *dst = L + blk * 2 * n2 * n2;           // [re|im][row][col]
    float m = 0.f;
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
        const float2 v = src[e];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmaxf(s, wm[w]);
    if (!(s > 0.f)) s = 1.f;
    const float inv = 1.f / s;
    for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
        const int col = e / n2, row = e % n2;
        const float2 v = src[e];
        dst[(size_t)row * n2 + col] = H16<H>::from(v.x * inv);
        dst[(size_t)n2 * n2 + (size_t)row * n2 + col] = H16<H>::from(v.y * inv);
    }
    if (threadIdx.x == 0) scale[blk] = s;
}

void compress_coarse(Ctx &c) {
    const int n2 = 2 * c.prm.n_tv;
    const size_t nblk = (size_t)9 * c.nagg;
    c.Dc16.alloc(nblk * 2 * n2 * n2 * sizeof(__half));
    c.Dcs.alloc(nblk * sizeof(float));
    TimeScope ts(c.timer, K_COARSE_BUILD, (double)nblk * n2 * n2 * (8 + 4));
    if (c.prm.coarse_links == MGEIG_LINKS_BF16)
        compress_coarse_kernel<__nv_bfloat16><<<(int)nblk, 256, 0, c.stream>>>(n2, c.Dc.as<float2>(),
                                                                              c.Dc16.as<__nv_bfloat16>(),
                                                                              c.Dcs.as<float>());
    else
        compress_coarse_kernel<__half><<<(int)nblk, 256, 0, c.stream>>>(n2, c.Dc.as<float2>(), c.Dc16.as<__half>(),
                                                                       c.Dcs.as<float>());
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// one right-hand side, FP32 arithmetic: thread per (coarse site, row)

template <typename H>
__global__ void coarse_apply16_kernel(int nagg, int ntv, const H *__restrict__ L, const float *__restrict__ scale,
                                      const int *__restrict__ nbr, float sigma, const float2 *__restrict__ x,
                                      float2 *__restrict__ y, int dform) {
    using HP = typename H16<H>::P;
    const int n2 = 2 * ntv;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nagg * n2) return;
    const int a = (int)(t / n2), row = (int)(t % n2);
    float ar = 0.f, ai = 0.f;
    for (int d = 0; d < 9; ++d) {
        const size_t blk = (size_t)d * nagg + a;
        const int b = __ldg(nbr + blk);
        const HP *pr = reinterpret_cast<const HP *>(L + blk * 2 * n2 * n2 + (size_t)row * n2);
        const HP *pi = reinterpret_cast<const HP *>(L + blk * 2 * n2 * n2 + (size_t)n2 * n2 + (size_t)row * n2);
        const float4 *xb = reinterpret_cast<const float4 *>(x + (size_t)b * n2);
        float dr = 0.f, di = 0.f;
        for (int p = 0; p < n2 / 2; ++p) {
            const float2 r = H16<H>::pair(pr[p]), im = H16<H>::pair(pi[p]);
            const float4 xv = xb[p];   // x_2p, x_2p+1
            dr = fmaf(r.x, xv.x, dr); dr = fmaf(-im.x, xv.y, dr);
            di = fmaf(r.x, xv.y, di); di = fmaf(im.x, xv.x, di);
            dr = fmaf(r.y, xv.z, dr); dr = fmaf(-im.y, xv.w, dr);
            di = fmaf(r.y, xv.w, di); di = fmaf(im.y, xv.z, di);
        }
        const float s = __ldg(scale + blk);
        ar = fmaf(s, dr, ar);
        ai = fmaf(s, di, ai);
    }
    const float2 xt = x[t];
    if (dform) {
        const float sg = row >= ntv ? -sigma : sigma;
        y[t] = make_float2(ar - sg * xt.x, ai - sg * xt.y);
    } else {
        if (row >= ntv) { ar = -ar; ai = -ai; }
        y[t] = make_float2(ar - sigma * xt.x, ai - sigma * xt.y);
    }
}

void coarse_apply_links16(Ctx &c, double sigma, const void *x, void *y, bool dform) {
    const int ntv = c.prm.n_tv, n2 = 2 * ntv;
    MG_REQUIRE(n2 % 2 == 0 && c.Dc16.p && c.cnbr.p, MGEIG_ENOTSETUP);
    const size_t n = (size_t)c.nagg * n2;
    TimeScope ts(c.timer, K_COARSE_APPLY, (double)c.nagg * (9.0 * (2 * n2 * n2 * 2 + 4) + 2.0 * n2 * 8));
    if (c.prm.coarse_links == MGEIG_LINKS_BF16)
        coarse_apply16_kernel<__nv_bfloat16><<<grid_for(n, 128), 128, 0, c.stream>>>(
            c.nagg, ntv, c.Dc16.as<__nv_bfloat16>(), c.Dcs.as<float>(), c.cnbr.as<int>(), (float)sigma,
            static_cast<const float2 *>(x), static_cast<float2 *>(y), dform ? 1 : 0);
    else
        coarse_apply16_kernel<__half><<<grid_for(n, 128), 128, 0, c.stream>>>(
            c.nagg, ntv, c.Dc16.as<__half>(), c.Dcs.as<float>(), c.cnbr.as<int>(), (float)sigma,
            static_cast<const float2 *>(x), static_cast<float2 *>(y), dform ? 1 : 0);
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// nrhs right-hand sides on the tensor cores (BF16 links)

constexpr int TC_WARPS = 6;                  // warp w: row tile w / 2, plane w % 2
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_MAXN = 16;                  // right-hand sides per launch
constexpr int TC_BP = 56;                    // staged B pitch (halves): conflict-free fragment reads
constexpr int TC_MAXNT = 2 * TC_MAXN / 8;    // n tiles of 8 columns
constexpr int TC_SLACK = 16 * 48 + 64;       // zero halves after the last plane (rows / columns to 48)

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// Shared memory of one CTA (one coarse site), n2 = 2 N_tv <= 48 rows:
//   As  a ring of two hop buffers: one link block's planes as stored in global
//       memory ([re|im][row][col], n2 x n2 each, row pitch n2 halves) plus TC_SLACK
//       zero halves (the row and column tiles run to the next multiple of 16, the
//       extra columns read finite entries of the next row that meet zero rows of
//       B, and the extra rows are dropped).  Hop d + 1 is copied (cp.async) while
//       hop d is multiplied
//   Bs  [d][column n < 8 NT][k < 48] staged s_d [Xr | Xi], zero for k >= n2
//   Cs  (after the products) [plane][48][2 nrhs] accumulators
__global__ void __launch_bounds__(TC_THREADS, 5)
coarse_apply_nrhs_tc_kernel(int nagg, int ntv, int nrhs, int NT, const __nv_bfloat16 *__restrict__ L,
                            const float *__restrict__ scale, const int *__restrict__ nbr, float sigma,
                            const float2 *__restrict__ X, float2 *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    const int n2 = 2 * ntv;
    const int site = blockIdx.x;
    const size_t plane = (size_t)n2 * n2;
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(tc_smem);
    const size_t hop_elems = ((2 * plane + TC_SLACK + 7) / 8) * 8;   // one ring buffer (16-byte multiple)
    __nv_bfloat16 *Bs = As + 2 * hop_elems;
    const int ncols = 8 * NT;
    // 1. the link block of hop d (contiguous 2 n2^2 halves) into ring buffer d & 1
    //    by 16-byte async copies, one commit group per hop
    const int chunks_per_blk = (int)(2 * plane * 2 / 16);
    auto copy_hop = [&](int d) {
        const __nv_bfloat16 *src = L + ((size_t)d * nagg + site) * 2 * plane;
        __nv_bfloat16 *dst = As + (size_t)(d & 1) * hop_elems;
        for (int q = threadIdx.x; q < chunks_per_blk; q += blockDim.x)
            cp_async16(dst + (size_t)q * 8, src + (size_t)q * 8);
        asm volatile("cp.async.commit_group;\n" ::);
    };
    copy_hop(0);
    for (int e = threadIdx.x; e < TC_SLACK; e += blockDim.x) {
        As[2 * plane + e] = __float2bfloat16_rn(0.f);
        As[hop_elems + 2 * plane + e] = __float2bfloat16_rn(0.f);
    }
    // 2. right-hand sides of the nine neighbours, scaled by the link's scale, in BF16:
    //    warp-strided over (hop d, right-hand side r), lanes over the rows k; one
    //    float2 load fills column r (real parts) and column nrhs + r (imaginary)
    {
        const int wq = threadIdx.x >> 5, lq = threadIdx.x & 31, nwq = blockDim.x >> 5;
        for (int dr = wq; dr < 9 * nrhs; dr += nwq) {
            const int d = dr / nrhs, r = dr - d * nrhs;
            const size_t blk = (size_t)d * nagg + site;
            const int b = __ldg(nbr + blk);
            const float sc = __ldg(scale + blk);
            const float2 *xr = X + ((size_t)r * nagg + b) * n2;
            __nv_bfloat16 *br = Bs + ((size_t)d * ncols + r) * TC_BP;
            __nv_bfloat16 *bi = Bs + ((size_t)d * ncols + nrhs + r) * TC_BP;
            for (int k = lq; k < 48; k += 32) {
                float2 xv = make_float2(0.f, 0.f);
                if (k < n2) xv = xr[k];
                br[k] = __float2bfloat16_rn(sc * xv.x);
                bi[k] = __float2bfloat16_rn(sc * xv.y);
            }
        }
        // the padding columns 2 nrhs .. 8 NT - 1 of every hop are zero
        const int npad = ncols - 2 * nrhs;
        for (int e = threadIdx.x; e < 9 * npad * 48; e += blockDim.x) {
            const int k = e % 48, q = e / 48, d = q / npad, col = 2 * nrhs + q % npad;
            Bs[((size_t)d * ncols + col) * TC_BP + k] = __float2bfloat16_rn(0.f);
        }
    }
    // 3. products: warp w takes rows 16 (w / 2) .. +15 of plane w % 2, every column tile
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int mt = w >> 1, pl = w & 1;
    float acc[TC_MAXNT][4];
#pragma unroll
    for (int j = 0; j < TC_MAXNT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int d = 0; d < 9; ++d) {
        // hop d + 1 streams in while hop d is multiplied
        if (d + 1 < 9) {
            copy_hop(d + 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();   // hop d (and, for d = 0, the staged B and the slack) visible to all
        if (16 * mt < n2) {
            const __nv_bfloat16 *Ap = As + (size_t)(d & 1) * hop_elems + (size_t)pl * plane;
            const __nv_bfloat16 *Bp = Bs + (size_t)d * ncols * TC_BP;
            for (int ks = 0; ks < 3 && 16 * ks < n2; ++ks) {
                uint32_t a[4];
                const int r0 = 16 * mt + g, c0 = 16 * ks + 2 * tq;
                a[0] = *reinterpret_cast<const uint32_t *>(Ap + (size_t)r0 * n2 + c0);
                a[1] = *reinterpret_cast<const uint32_t *>(Ap + (size_t)(r0 + 8) * n2 + c0);
                a[2] = *reinterpret_cast<const uint32_t *>(Ap + (size_t)r0 * n2 + c0 + 8);
                a[3] = *reinterpret_cast<const uint32_t *>(Ap + (size_t)(r0 + 8) * n2 + c0 + 8);
#pragma unroll
                for (int j = 0; j < TC_MAXNT; ++j) {
                    if (j < NT) {
                        uint32_t b[2];
                        const __nv_bfloat16 *bc = Bp + (size_t)(8 * j + g) * TC_BP + 16 * ks + 2 * tq;
                        b[0] = *reinterpret_cast<const uint32_t *>(bc);
                        b[1] = *reinterpret_cast<const uint32_t *>(bc + 8);
                        mma_bf16_16816(acc[j], a, b);
                    }
                }
            }
        }
        __syncthreads();   // every read of ring buffer d & 1 is done before hop d + 2 overwrites it
    }
    // every read of As / Bs is done (the last barrier of the loop): the accumulators reuse the space
    float *Cs = reinterpret_cast<float *>(tc_smem);   // [plane][48][ncols]
    if (16 * mt < n2) {
#pragma unroll
        for (int j = 0; j < TC_MAXNT; ++j) {
            if (j < NT) {
                const int r = 16 * mt + g, col = 8 * j + 2 * tq;
                float *cp = Cs + (size_t)pl * 48 * ncols;
                cp[(size_t)r * ncols + col] = acc[j][0];
                cp[(size_t)r * ncols + col + 1] = acc[j][1];
                cp[(size_t)(r + 8) * ncols + col] = acc[j][2];
                cp[(size_t)(r + 8) * ncols + col + 1] = acc[j][3];
            }
        }
    }
    __syncthreads();
    // 4. Yr = Ar Xr - Ai Xi, Yi = Ar Xi + Ai Xr; then gamma5^c and the shift
    const float *Cr = Cs, *Ci = Cs + (size_t)48 * ncols;
    for (int e = threadIdx.x; e < nrhs * n2; e += blockDim.x) {
        const int row = e % n2, r = e / n2;
        float yr = Cr[(size_t)row * ncols + r] - Ci[(size_t)row * ncols + nrhs + r];
        float yi = Cr[(size_t)row * ncols + nrhs + r] + Ci[(size_t)row * ncols + r];
        if (row >= ntv) { yr = -yr; yi = -yi; }
        const size_t idx = ((size_t)r * nagg + site) * n2 + row;
        const float2 xv = X[idx];
        Y[idx] = make_float2(yr - sigma * xv.x, yi - sigma * xv.y);
    }
}

size_t coarse_nrhs_tc_smem(int n2, int NT) {
    const size_t hop_elems = ((2 * (size_t)n2 * n2 + TC_SLACK + 7) / 8) * 8;
    const size_t a = 2 * hop_elems * 2;
    const size_t b = (size_t)9 * 8 * NT * TC_BP * 2;
    const size_t cbytes = (size_t)2 * 48 * 8 * NT * 4;
    return std::max(a + b, cbytes);
}

void coarse_apply_nrhs(Ctx &c, double sigma, const void *X, void *Y, int nrhs) {
    const int ntv = c.prm.n_tv, n2 = 2 * ntv;
    MG_REQUIRE(nrhs >= 1 && nrhs <= TC_MAXN, MGEIG_EINVAL);
    MG_REQUIRE(c.cnbr.p && c.Dc.p, MGEIG_ENOTSETUP);
    const size_t vb = (size_t)c.nagg * n2 * sizeof(float2);
    if (c.prm.coarse_links != MGEIG_LINKS_BF16) {
        // FP32 or FP16 links: the CUDA-core kernels, one right-hand side after another
        for (int r = 0; r < nrhs; ++r) {
            const void *xr = static_cast<const char *>(X) + vb * r;
            void *yr = static_cast<char *>(Y) + vb * r;
            if (c.prm.coarse_links == MGEIG_LINKS_F16) coarse_apply_links16(c, sigma, xr, yr, false);
            else coarse_apply<float>(c, c.Dc.p, sigma, xr, yr, false);
        }
        return;
    }
    MG_REQUIRE(n2 <= 48 && c.Dc16.p, MGEIG_EINVAL);
    const int NT = (2 * nrhs + 7) / 8;
    const size_t smem = coarse_nrhs_tc_smem(n2, NT);
    MG_CUDA(cudaFuncSetAttribute(coarse_apply_nrhs_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    // algorithmic bytes: the 16-bit links and scales once, every right-hand side read
    // (nine neighbours from L2, counted once) and written once
    TimeScope ts(c.timer, K_COARSE_APPLY,
                 (double)c.nagg * (9.0 * (2 * n2 * n2 * 2 + 4) + (double)nrhs * 2 * n2 * 8));
    coarse_apply_nrhs_tc_kernel<<<c.nagg, TC_THREADS, smem, c.stream>>>(
        c.nagg, ntv, nrhs, NT, c.Dc16.as<__nv_bfloat16>(), c.Dcs.as<float>(), c.cnbr.as<int>(), (float)sigma,
        static_cast<const float2 *>(X), static_cast<float2 *>(Y));
    MG_CHECK_LAUNCH();
}

}  // namespace mgeig
