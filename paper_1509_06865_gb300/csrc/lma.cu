// Kernels of approximate low-mode averaging (Sec. 3.1 and 3.2): per-timeslice
// inner products of the kept approximate eigenvectors, from which the host forms
// the low-mode part of the disconnected loop
//     L_low(t) = sum_ij (A^-1)_ij sum_{x in t} <v_j(x) | v_i(x)>,
// the per-timeslice stochastic estimate of its high-mode part
//     L_high(t) = 1/N sum_n sum_{x in t} <eta_n(x) | s_n(x)>,  Q s_n = R~ eta_n,
// and Z2 + iZ2 noise fields (entries (+-1 +- i)/sqrt 2 from Philox sign bits,
// the generator of the seeded inputs: counter (site, component pair, field, tag)).
#include "internal.h"

namespace mgeig {

constexpr int TS_THREADS = 256;
constexpr int TS_CHUNK = 8;   // vectors i per block

// M[t][j][i] = sum_{x in timeslice t} <X_j(x) | Y_i(x)> (FP64 internal spinors,
// [12][V] each; a timeslice is a contiguous run of V3 sites); grid (T, nj, ceil(ni / 8))
__global__ void __launch_bounds__(TS_THREADS) timeslice_dots_kernel(int V, int V3, int nj, int ni,
                                                                    const double2 *const *X, const double2 *const *Y,
                                                                    double2 *M) {
    const int t = blockIdx.x, j = blockIdx.y, i0 = blockIdx.z * TS_CHUNK;
    const int cnt = min(TS_CHUNK, ni - i0);
    const double2 *xj = X[j];
    double re[TS_CHUNK], im[TS_CHUNK];
#pragma unroll
    for (int q = 0; q < TS_CHUNK; ++q) { re[q] = 0; im[q] = 0; }
    for (int e = threadIdx.x; e < 12 * V3; e += blockDim.x) {
        const int k = e / V3, s = t * V3 + e % V3;
        const double2 a = xj[(size_t)k * V + s];
#pragma unroll
        for (int q = 0; q < TS_CHUNK; ++q) {
            if (q < cnt) {
                const double2 b = Y[i0 + q][(size_t)k * V + s];
                re[q] = fma(a.x, b.x, re[q]); re[q] = fma(a.y, b.y, re[q]);
                im[q] = fma(a.x, b.y, im[q]); im[q] = fma(-a.y, b.x, im[q]);
            }
        }
    }
    __shared__ double sh[TS_THREADS / 32][2 * TS_CHUNK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < TS_CHUNK; ++q) {
        double a = re[q], b = im[q];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { sh[w][2 * q] = a; sh[w][2 * q + 1] = b; }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double a = 0, b = 0;
        for (int ww = 0; ww < TS_THREADS / 32; ++ww) { a += sh[ww][2 * threadIdx.x]; b += sh[ww][2 * threadIdx.x + 1]; }
        M[((size_t)t * nj + j) * ni + i0 + threadIdx.x] = make_double2(a, b);
    }
}

void timeslice_dots(Ctx &c, const void *const *X, int nj, const void *const *Y, int ni, void *M_dev) {
    const int T = c.dims[3], V3 = c.g.V / T;
    TmpBuf ptrs;
    ptrs.alloc((size_t)(nj + ni) * sizeof(void *));
    std::vector<const void *> h(X, X + nj);
    h.insert(h.end(), Y, Y + ni);
    MG_CUDA(cudaMemcpyAsync(ptrs.p, h.data(), h.size() * sizeof(void *), cudaMemcpyHostToDevice, c.stream));
    const double2 *const *Xd = ptrs.as<const double2 *>();
    TimeScope ts(c.timer, K_BLAS_F64, (double)(nj + (double)nj * ni / TS_CHUNK) * c.fine_ncpx() * 16);
    timeslice_dots_kernel<<<dim3(T, nj, (ni + TS_CHUNK - 1) / TS_CHUNK), TS_THREADS, 0, c.stream>>>(
        c.g.V, V3, nj, ni, Xd, Xd + nj, static_cast<double2 *>(M_dev));
    MG_CHECK_LAUNCH();
    sync(c);   // the pointer table is freed on return
}

__device__ __forceinline__ void philox4x32_10_lma(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// Z2 + iZ2 noise: the sign bit of each Philox word, value +-1/sqrt 2
__global__ void z2_spinor_kernel(int V, int n, uint32_t k0, uint32_t k1, uint32_t tag, double2 *__restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * n * 6) return;
    const int q = (int)(i % 6);
    const int s = (int)((i / 6) % V);
    const int j = (int)(i / ((size_t)6 * V));
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)q, (uint32_t)j, tag};
    philox4x32_10_lma(ctr, k0, k1);
    const double h = 0.70710678118654752440;
    double2 *o = out + (size_t)j * 12 * V;
    o[(size_t)(2 * q) * V + s] = make_double2(ctr[0] >> 31 ? -h : h, ctr[1] >> 31 ? -h : h);
    o[(size_t)(2 * q + 1) * V + s] = make_double2(ctr[2] >> 31 ? -h : h, ctr[3] >> 31 ? -h : h);
}

void z2_spinors(Ctx &c, uint64_t seed, void *out64, int n, uint32_t tag) {
    const size_t tot = (size_t)c.g.V * n * 6;
    z2_spinor_kernel<<<grid_for(tot, 256), 256, 0, c.stream>>>(c.g.V, n, (uint32_t)(seed & 0xFFFFFFFFu),
                                                               (uint32_t)(seed >> 32), tag,
                                                               static_cast<double2 *>(out64));
    MG_CHECK_LAUNCH();
}

}  // namespace mgeig
