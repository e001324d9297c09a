// Focal-length vote (Sec. "Intrinsics Estimation", paragraph "Focal Length Estimation",
// Eq. fastmap-focal-vote): a 3x3 matrix is an essential matrix exactly when its two largest
// singular values are equal and the third is zero, so a candidate focal length f is scored over
// the image pairs i by
//     v(f) = sum_i exp((1 - lambda_1 / lambda_2) / tau),   lambda of E_i = K_2^T F_i K_1,
// K = diag(f, f, 1) (principal point at the image centre). A side of a pair whose focal length
// is already known uses it instead of the candidate (the paper's several-camera procedure).
//
// One thread evaluates one (candidate, pair) term: E from F (FP32, F normalised to unit
// Frobenius norm on the host, which leaves the ratio unchanged), M = E^T E, its eigenvalues by
// four sweeps of cyclic Jacobi rotations (each 2x2 step uses the cancellation-free rotation
// angle, so nearly equal eigenvalues keep their relative accuracy, unlike the closed-form cubic
// roots), lambda_1 / lambda_2 = sqrt(mu_1 / mu_2). A block covers 256 pairs and VOTE_CANDS
// candidates; per-block sums are reduced in a fixed order, then added per candidate in FP64 in
// block order: the votes are bit-reproducible.
#include <cmath>
#include <string>
#include <vector>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int VOTE_THREADS = 256;
constexpr int VOTE_CANDS = 16;
constexpr int JACOBI_SWEEPS = 4;

// one Jacobi rotation of the symmetric 3x3 matrix (a00, a11, a22, a01, a02, a12) in plane (p, q)
__device__ __forceinline__ void jacobi_rot(float &app, float &aqq, float &apq, float &arp, float &arq) {
    if (apq == 0.f) return;
    const float theta = (aqq - app) / (2.f * apq);
    const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
    const float c = rsqrtf(fmaf(t, t, 1.f)), s = t * c;
    app = fmaf(-t, apq, app);
    aqq = fmaf(t, apq, aqq);
    apq = 0.f;
    const float rp = arp, rq = arq;
    arp = c * rp - s * rq;
    arq = s * rp + c * rq;
}

__device__ __forceinline__ float vote_term(const float *F, float f1, float f2, float inv_tau) {
    const float s1[3] = {f1, f1, 1.f}, s2[3] = {f2, f2, 1.f};
    float E[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) E[3 * a + b] = (s2[a] * F[3 * a + b]) * s1[b];
    // M = E^T E
    float m00 = 0.f, m11 = 0.f, m22 = 0.f, m01 = 0.f, m02 = 0.f, m12 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e0 = E[3 * a], e1 = E[3 * a + 1], e2 = E[3 * a + 2];
        m00 = fmaf(e0, e0, m00);
        m11 = fmaf(e1, e1, m11);
        m22 = fmaf(e2, e2, m22);
        m01 = fmaf(e0, e1, m01);
        m02 = fmaf(e0, e2, m02);
        m12 = fmaf(e1, e2, m12);
    }
#pragma unroll
    for (int sweep = 0; sweep < JACOBI_SWEEPS; ++sweep) {
        jacobi_rot(m00, m11, m01, m02, m12);   // plane (0, 1); third index 2
        jacobi_rot(m00, m22, m02, m01, m12);   // plane (0, 2); third index 1
        jacobi_rot(m11, m22, m12, m01, m02);   // plane (1, 2); third index 0
    }
    // the two largest of the eigenvalues (clamped at 0: M is positive semi-definite)
    const float e0 = fmaxf(m00, 0.f), e1 = fmaxf(m11, 0.f), e2 = fmaxf(m22, 0.f);
    const float hi = fmaxf(e0, fmaxf(e1, e2));
    const float lo = fminf(e0, fminf(e1, e2));
    const float mid = (e0 + e1 + e2) - hi - lo;
    if (!(mid > 0.f)) return 0.f;
    const float ratio = sqrtf(hi / mid);
    return expf((1.f - ratio) * inv_tau);
}

// grid (pair blocks, candidate chunks); partial[c * n_blocks + block] for candidate c
__global__ void __launch_bounds__(VOTE_THREADS)
k_focal_vote(const float *F, const float *f1k, const float *f2k, int n_pairs, const float *cand, int n_cand,
             float inv_tau, float *partial) {
    __shared__ float red[VOTE_CANDS][VOTE_THREADS / 32];
    const int n = blockIdx.x * VOTE_THREADS + threadIdx.x;
    const int c0 = blockIdx.y * VOTE_CANDS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float Fn[9];
    float k1 = 0.f, k2 = 0.f;
    const bool valid = n < n_pairs;
    if (valid) {
#pragma unroll
        for (int q = 0; q < 9; ++q) Fn[q] = F[(size_t)n * 9 + q];
        k1 = f1k ? f1k[n] : 0.f;
        k2 = f2k ? f2k[n] : 0.f;
    }
#pragma unroll 1
    for (int cc = 0; cc < VOTE_CANDS; ++cc) {
        const int c = c0 + cc;
        float v = 0.f;
        if (valid && c < n_cand) {
            const float f = cand[c];
            v = vote_term(Fn, k1 > 0.f ? k1 : f, k2 > 0.f ? k2 : f, inv_tau);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[cc][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < VOTE_CANDS) {
        const int c = c0 + threadIdx.x;
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < VOTE_THREADS / 32; ++w) s += red[threadIdx.x][w];
        if (c < n_cand) partial[(size_t)c * gridDim.x + blockIdx.x] = s;
    }
}

// one warp per candidate: FP64 sum of its block partials in block order
__global__ void k_focal_vote_sum(const float *partial, int n_blocks, int n_cand, double *votes) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_cand) return;
    double s = 0.0;
    for (int b = lane; b < n_blocks; b += 32) s += (double)partial[(size_t)c * n_blocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) votes[c] = s;
}

}  // namespace
}  // namespace fm

using namespace fm;

void fm_internal_set_error(const char *msg);

namespace {
fm_status fv_fail(fm_status s, const std::string &m) {
    fm_internal_set_error(("fm_focal_vote: " + m).c_str());
    return s;
}
}  // namespace

extern "C" FM_API fm_status fm_focal_vote(int32_t n_pairs, const double *F, const double *f1_known,
                                          const double *f2_known, int32_t n_cand, const double *cand,
                                          double tau, double *votes, float *elapsed_ms, void *stream) {
    if (n_pairs < 1 || n_cand < 1) return fv_fail(FM_EINVAL, "n_pairs and n_cand must be >= 1");
    if ((int64_t)n_cand > 65535LL * VOTE_CANDS) return fv_fail(FM_EINVAL, "n_cand must be <= 1048560");
    if (!F || !cand || !votes) return fv_fail(FM_EINVAL, "F, cand and votes must not be NULL");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fv_fail(FM_EINVAL, "tau must be finite and > 0");
    std::vector<float> hF((size_t)n_pairs * 9), hk1, hk2, hc(n_cand);
    for (int n = 0; n < n_pairs; ++n) {
        double nrm = 0.0;
        for (int q = 0; q < 9; ++q) {
            const double v = F[(size_t)n * 9 + q];
            if (!std::isfinite(v)) return fv_fail(FM_EINVAL, "F must be finite");
            nrm += v * v;
        }
        if (!(nrm > 0.0)) return fv_fail(FM_EINVAL, "F of pair " + std::to_string(n) + " is zero");
        const double inv = 1.0 / std::sqrt(nrm);
        for (int q = 0; q < 9; ++q) hF[(size_t)n * 9 + q] = (float)(F[(size_t)n * 9 + q] * inv);
    }
    auto known = [&](const double *src, std::vector<float> &dst) -> bool {
        if (!src) return true;
        dst.resize(n_pairs);
        for (int n = 0; n < n_pairs; ++n) {
            if (!(src[n] >= 0.0) || !std::isfinite(src[n])) return false;
            dst[n] = (float)src[n];
        }
        return true;
    };
    if (!known(f1_known, hk1) || !known(f2_known, hk2))
        return fv_fail(FM_EINVAL, "known focal lengths must be finite and >= 0 (0 = the candidate)");
    for (int c = 0; c < n_cand; ++c) {
        if (!(cand[c] > 0.0) || !std::isfinite(cand[c])) return fv_fail(FM_EINVAL, "candidates must be finite and > 0");
        hc[c] = (float)cand[c];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_blocks = (n_pairs + VOTE_THREADS - 1) / VOTE_THREADS;
    const int n_chunks = (n_cand + VOTE_CANDS - 1) / VOTE_CANDS;
    float *dF = nullptr, *dk1 = nullptr, *dk2 = nullptr, *dc = nullptr, *dpart = nullptr;
    double *dv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    step(cudaMallocAsync(&dF, sizeof(float) * hF.size(), s));
    if (!hk1.empty()) step(cudaMallocAsync(&dk1, sizeof(float) * n_pairs, s));
    if (!hk2.empty()) step(cudaMallocAsync(&dk2, sizeof(float) * n_pairs, s));
    step(cudaMallocAsync(&dc, sizeof(float) * n_cand, s));
    step(cudaMallocAsync(&dpart, sizeof(float) * (size_t)n_blocks * n_cand, s));
    step(cudaMallocAsync(&dv, sizeof(double) * n_cand, s));
    step(cudaMemcpyAsync(dF, hF.data(), sizeof(float) * hF.size(), cudaMemcpyHostToDevice, s));
    if (dk1) step(cudaMemcpyAsync(dk1, hk1.data(), sizeof(float) * n_pairs, cudaMemcpyHostToDevice, s));
    if (dk2) step(cudaMemcpyAsync(dk2, hk2.data(), sizeof(float) * n_pairs, cudaMemcpyHostToDevice, s));
    step(cudaMemcpyAsync(dc, hc.data(), sizeof(float) * n_cand, cudaMemcpyHostToDevice, s));
    if (elapsed_ms) {
        step(cudaEventCreate(&e0));
        step(cudaEventCreate(&e1));
        if (e == cudaSuccess) step(cudaEventRecord(e0, s));
    }
    if (e == cudaSuccess) {
        k_focal_vote<<<dim3(n_blocks, n_chunks), VOTE_THREADS, 0, s>>>(dF, dk1, dk2, n_pairs, dc, n_cand,
                                                                      (float)(1.0 / tau), dpart);
        k_focal_vote_sum<<<(n_cand + 7) / 8, 256, 0, s>>>(dpart, n_blocks, n_cand, dv);
        step(cudaGetLastError());
    }
    if (elapsed_ms && e == cudaSuccess) step(cudaEventRecord(e1, s));
    if (e == cudaSuccess) step(cudaMemcpyAsync(votes, dv, sizeof(double) * n_cand, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(dF, s);
    if (dk1) cudaFreeAsync(dk1, s);
    if (dk2) cudaFreeAsync(dk2, s);
    cudaFreeAsync(dc, s);
    cudaFreeAsync(dpart, s);
    cudaFreeAsync(dv, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    if (elapsed_ms && e == cudaSuccess) e = cudaEventElapsedTime(elapsed_ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess)
        return fv_fail(e == cudaErrorMemoryAllocation ? FM_ENOMEM : FM_ECUDA, cudaGetErrorString(e));
    return FM_OK;
}
