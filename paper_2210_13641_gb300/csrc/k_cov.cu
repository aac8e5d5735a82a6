// k_cov.cu - marginal covariances of the tracking frontend's dense bundle
// adjustment, the producer of the per-pixel depth variances Sigma_D that weight the
// mapping loss (Sec. 3.1, Eq. cov).  The BA Hessian has the cameras/depths arrow
// structure H = [[C, E], [E^T, P]] (Eq. hessian): C the 6K x 6K camera block, P
// diagonal (one inverse depth per pixel), E block-sparse (per pixel, the 6-vectors
// of the few poses its flow residuals involve).  Then
//   H_T = C - E P^-1 E^T = L L^T,   Sigma_T = (L L^T)^-1,
//   Sigma_d = diag(P^-1 + P^-T E^T Sigma_T E P^-1).
// FP64 throughout: the reduced camera matrix of a bundle adjustment is badly
// conditioned, and the work is small (the camera block of a keyframe window has at
// most kCovMaxC rows).
//   k_cov_schur   pixels -> sum_q e_a e_b^T / P_q into a shared-memory copy of the
//                 c x c matrix per block, flushed with FP64 atomics;
//   k_cov_chol    one block: C - that sum, Cholesky (packed lower triangle in shared
//                 memory), L^-1 by forward substitution, Sigma_T = L^-T L^-1;
//   k_cov_depth   one thread per pixel: 1/P + (E P^-1)_q^T Sigma_T (E P^-1)_q.
#include <cstdint>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "nerfmap.h"
#include "internal.h"

namespace nm {

namespace {

constexpr uint32_t kCovMaxC = 144;  // 24 keyframes
constexpr uint32_t kCovMaxB = 8;
constexpr int kCovThreads = 1024;

void set_cov_error(const char* msg) { set_global_error(msg); }

__device__ __forceinline__ uint32_t tri(uint32_t i, uint32_t j) { return i * (i + 1) / 2 + j; }  // i >= j

// Per block: the pixels q = blockIdx.x, blockIdx.x + gridDim.x, ... (one warp per
// pixel) add e_a e_b^T / P_q for every pair of its blocks (a, b) to a shared copy of
// the c x c matrix (lower triangle, packed), which is then added to acc.
__global__ void __launch_bounds__(256) k_cov_schur(uint32_t c, const double* __restrict__ P, uint32_t p,
                                                   const int32_t* __restrict__ blk, const double* __restrict__ e,
                                                   uint32_t B, double* __restrict__ acc, uint32_t* __restrict__ flag) {
    extern __shared__ double sh[];
    const uint32_t n_tri = c * (c + 1) / 2;
    for (uint32_t i = threadIdx.x; i < n_tri; i += blockDim.x) sh[i] = 0.0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warps = blockDim.x >> 5;
    const uint32_t n_entries = B * B * 36;
    for (uint32_t q = blockIdx.x * warps + (threadIdx.x >> 5); q < p; q += gridDim.x * warps) {
        const double Pq = P[q];
        if (!(Pq > 0.0)) {
            if (lane == 0) atomicOr(flag, 1u);
            continue;
        }
        const double inv = 1.0 / Pq;
        for (uint32_t t = lane; t < n_entries; t += 32) {
            const uint32_t ab = t / 36, rc = t % 36;
            const uint32_t a = ab / B, b = ab % B, r = rc / 6, col = rc % 6;
            const int32_t ka = blk[(size_t)q * B + a], kb = blk[(size_t)q * B + b];
            if (ka < 0 || kb < 0) continue;
            const uint32_t i = 6u * (uint32_t)ka + r, j = 6u * (uint32_t)kb + col;
            if (i < j || i >= c) continue;  // lower triangle (the pair (b, a) covers the rest)
            atomicAdd(&sh[tri(i, j)], e[((size_t)q * B + a) * 6 + r] * e[((size_t)q * B + b) * 6 + col] * inv);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_tri; i += blockDim.x)
        if (sh[i] != 0.0) atomicAdd(&acc[i], sh[i]);
}

// One block: H_T = C - acc (packed lower), Cholesky in place, Y = L^-1 (packed
// lower, forward substitution per column), Sigma_T = Y^T Y (full c x c, row-major).
__global__ void __launch_bounds__(kCovThreads) k_cov_chol(uint32_t c, const double* __restrict__ C,
                                                          const double* __restrict__ acc, double* __restrict__ ST,
                                                          uint32_t* __restrict__ flag) {
    extern __shared__ double sh[];
    const uint32_t n_tri = c * (c + 1) / 2;
    double* A = sh;          // packed lower: H_T, then L
    double* Y = sh + n_tri;  // packed lower: L^-1
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (uint32_t t = threadIdx.x; t < n_tri; t += blockDim.x) {
        // row i, column j of the packed index t
        uint32_t i = (uint32_t)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while (tri(i, 0) > t) --i;
        while (tri(i + 1, 0) <= t) ++i;
        const uint32_t j = t - tri(i, 0);
        A[t] = C[(size_t)i * c + j] - acc[t];
    }
    __syncthreads();
    // right-looking Cholesky
    for (uint32_t j = 0; j < c; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[tri(j, j)];
            if (!(d > 0.0)) bad = 1;
            A[tri(j, j)] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double ljj = A[tri(j, j)];
        for (uint32_t i = j + 1 + threadIdx.x; i < c; i += blockDim.x) A[tri(i, j)] /= ljj;
        __syncthreads();
        const uint32_t m = c - j - 1;  // trailing size
        for (uint32_t t = threadIdx.x; t < m * (m + 1) / 2; t += blockDim.x) {
            uint32_t ii = (uint32_t)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while (tri(ii, 0) > t) --ii;
            while (tri(ii + 1, 0) <= t) ++ii;
            const uint32_t kk = t - tri(ii, 0);
            const uint32_t i = j + 1 + ii, k = j + 1 + kk;
            A[tri(i, k)] -= A[tri(i, j)] * A[tri(k, j)];
        }
        __syncthreads();
    }
    // Y = L^-1: column j by forward substitution (one thread per column)
    for (uint32_t j = threadIdx.x; j < c; j += blockDim.x) {
        Y[tri(j, j)] = 1.0 / A[tri(j, j)];
        for (uint32_t i = j + 1; i < c; ++i) {
            double s = 0.0;
            for (uint32_t k = j; k < i; ++k) s += A[tri(i, k)] * Y[tri(k, j)];
            Y[tri(i, j)] = -s / A[tri(i, i)];
        }
    }
    __syncthreads();
    // Sigma_T = Y^T Y: (i, j) = sum_{k >= max(i, j)} Y[k][i] Y[k][j]
    for (uint32_t t = threadIdx.x; t < c * c; t += blockDim.x) {
        const uint32_t i = t / c, j = t % c;
        double s = 0.0;
        for (uint32_t k = (i > j ? i : j); k < c; ++k) s += Y[tri(k, i)] * Y[tri(k, j)];
        ST[t] = s;
    }
    if (threadIdx.x == 0 && bad) atomicOr(flag, 2u);
}

// Per pixel: Sigma_d = 1/P + (E P^-1)_q^T Sigma_T (E P^-1)_q over its blocks.
__global__ void k_cov_depth(uint32_t c, const double* __restrict__ P, uint32_t p, const int32_t* __restrict__ blk,
                            const double* __restrict__ e, uint32_t B, const double* __restrict__ ST,
                            double* __restrict__ Sd) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p) return;
    const double inv = 1.0 / P[q];
    double s = 0.0;
    for (uint32_t a = 0; a < B; ++a) {
        const int32_t ka = blk[(size_t)q * B + a];
        if (ka < 0 || 6u * (uint32_t)ka >= c) continue;
        for (uint32_t b = 0; b < B; ++b) {
            const int32_t kb = blk[(size_t)q * B + b];
            if (kb < 0 || 6u * (uint32_t)kb >= c) continue;
            for (uint32_t r = 0; r < 6; ++r) {
                const double ea = e[((size_t)q * B + a) * 6 + r];
                const double* row = ST + (size_t)(6u * (uint32_t)ka + r) * c + 6u * (uint32_t)kb;
                double t = 0.0;
                for (uint32_t col = 0; col < 6; ++col) t += row[col] * e[((size_t)q * B + b) * 6 + col];
                s += ea * t;
            }
        }
    }
    Sd[q] = inv + s * inv * inv;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

}  // namespace nm

using namespace nm;

extern "C" int map_marginal_covariances(const double* C, uint32_t c, const double* P, uint32_t p,
                                        const int32_t* blk, const double* e, uint32_t B, double* sigma_T,
                                        double* sigma_d, int mem_kind, void* stream) {
    clear_global_error();
    if (!C || !P || !blk || !e || !sigma_T || !sigma_d) {
        set_cov_error("map_marginal_covariances: null argument");
        return MAP_EINVAL;
    }
    if (c == 0 || c % 6 != 0 || c > kCovMaxC || B == 0 || B > kCovMaxB || p == 0) {
        set_cov_error("map_marginal_covariances: need c = 6..144 (a multiple of 6), 1 <= B <= 8, p >= 1");
        return MAP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool host = mem_kind != MAP_MEM_DEVICE;
    const size_t bC = (size_t)c * c * sizeof(double), bP = (size_t)p * sizeof(double);
    const size_t bBlk = (size_t)p * B * sizeof(int32_t), bE = (size_t)p * B * 6 * sizeof(double);
    const size_t n_tri = (size_t)c * (c + 1) / 2;
    DevBuf work, inputs;
    // work: acc (packed), flag
    if (cudaMalloc(&work.p, n_tri * sizeof(double) + 16) != cudaSuccess) {
        set_cov_error("map_marginal_covariances: cudaMalloc failed");
        return MAP_ENOMEM;
    }
    double* acc = static_cast<double*>(work.p);
    uint32_t* flag = reinterpret_cast<uint32_t*>(acc + n_tri);
    const double *dC = C, *dP = P, *dE = e;
    const int32_t* dBlk = blk;
    double *dST = sigma_T, *dSd = sigma_d;
    if (host) {
        if (cudaMalloc(&inputs.p, bC + bP + bBlk + bE + bC + bP + 64) != cudaSuccess) {
            set_cov_error("map_marginal_covariances: cudaMalloc failed");
            return MAP_ENOMEM;
        }
        char* q = static_cast<char*>(inputs.p);
        double* hC = reinterpret_cast<double*>(q);
        double* hP = reinterpret_cast<double*>(q + bC);
        double* hE = reinterpret_cast<double*>(q + bC + bP);
        int32_t* hB = reinterpret_cast<int32_t*>(q + bC + bP + bE);
        double* hST = reinterpret_cast<double*>(q + bC + bP + bE + ((bBlk + 7) / 8) * 8);
        double* hSd = hST + (size_t)c * c;
        if (cudaMemcpyAsync(hC, C, bC, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(hP, P, bP, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(hE, e, bE, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(hB, blk, bBlk, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            set_cov_error("map_marginal_covariances: copy to the device failed");
            return MAP_ECUDA;
        }
        dC = hC;
        dP = hP;
        dE = hE;
        dBlk = hB;
        dST = hST;
        dSd = hSd;
    }
    cudaMemsetAsync(work.p, 0, n_tri * sizeof(double) + 16, s);
    const size_t sh_schur = n_tri * sizeof(double), sh_chol = 2 * n_tri * sizeof(double);
    // per call: the attribute belongs to the current device (cheap next to the kernel)
    cudaFuncSetAttribute(k_cov_schur, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kCovMaxC * (kCovMaxC + 1) / 2 * sizeof(double)));
    cudaFuncSetAttribute(k_cov_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kCovMaxC * (kCovMaxC + 1) * sizeof(double)));
    uint32_t grid = (p + 7) / 8;
    if (grid > 152u * 2u) grid = 152u * 2u;
    k_cov_schur<<<grid, 256, sh_schur, s>>>(c, dP, p, dBlk, dE, B, acc, flag);
    k_cov_chol<<<1, kCovThreads, sh_chol, s>>>(c, dC, acc, dST, flag);
    k_cov_depth<<<(p + 255) / 256, 256, 0, s>>>(c, dP, p, dBlk, dE, B, dST, dSd);
    if (cudaGetLastError() != cudaSuccess) {
        set_cov_error("map_marginal_covariances: kernel launch failed");
        return MAP_ECUDA;
    }
    uint32_t hflag = 0;
    if (host) {
        if (cudaMemcpyAsync(sigma_T, dST, bC, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(sigma_d, dSd, bP, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            set_cov_error("map_marginal_covariances: copy to the host failed");
            return MAP_ECUDA;
        }
    }
    if (cudaMemcpyAsync(&hflag, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_cov_error("map_marginal_covariances: device error");
        return MAP_ECUDA;
    }
    if (hflag & 1u) {
        set_cov_error("map_marginal_covariances: a pixel's P entry is not positive");
        return MAP_EINVAL;
    }
    if (hflag & 2u) {
        set_cov_error("map_marginal_covariances: the reduced camera matrix is not positive definite");
        return MAP_EINVAL;
    }
    return MAP_OK;
}
