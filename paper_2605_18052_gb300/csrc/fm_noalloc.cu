// Loss and gradient for callers that cannot allocate device memory.
//
// fm_create_problem owns its buffers and calls cudaMalloc; some callers cannot: code running
// under a memory manager that owns every byte of device memory (a framework's caching
// allocator, a fixed arena), or a latency-bound loop where cudaMalloc's implicit device
// synchronisation is not acceptable. fm_loss_grad_noalloc serves them: the caller passes its
// own device inputs and outputs, and every intermediate buffer (camera records, pair
// geometry, per-range partial sums, per-pair gradients, camera lists) lives in one
// file-scope __device__ array of fixed size. Nothing here calls cudaMalloc, cudaFree or any
// allocating library routine.
//
// The array belongs to every device that loads this library and stays there until the
// process exits. Its device address is looked up once per device (cudaGetSymbolAddress with
// that device current) on the first call made on that device.
#include <mutex>

#include "fm_internal.cuh"

namespace fm {
namespace {

constexpr int NA_MAX_CAMS = 4096;
constexpr int NA_MAX_PAIRS = 32768;
constexpr int64_t NA_MAX_PP = (int64_t)1 << 26;
constexpr int NA_MAX_RANGES = (int)(NA_MAX_PP / WR);

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_CAM = 0;
constexpr size_t OFF_CEN = OFF_CAM + al256(sizeof(float) * CAMREC * NA_MAX_CAMS);
constexpr size_t OFF_GEO = OFF_CEN + al256(sizeof(float2) * NA_MAX_CAMS);
constexpr size_t OFF_RANGE = OFF_GEO + al256(sizeof(float) * GEO * NA_MAX_PAIRS);
constexpr size_t OFF_SLOTS = OFF_RANGE + al256(sizeof(int) * NA_MAX_RANGES);
constexpr size_t OFF_PG = OFF_SLOTS + al256(sizeof(float) * SLOT * ((size_t)NA_MAX_PAIRS + NA_MAX_RANGES));
constexpr size_t OFF_CAMOFF = OFF_PG + al256(sizeof(float) * PG * NA_MAX_PAIRS);
constexpr size_t OFF_CAMENT = OFF_CAMOFF + al256(sizeof(int) * (NA_MAX_CAMS + 1));
constexpr size_t OFF_CAMTMP = OFF_CAMENT + al256(sizeof(int) * 2 * NA_MAX_PAIRS);
constexpr size_t OFF_CURSOR = OFF_CAMTMP + al256(sizeof(int) * 2 * NA_MAX_PAIRS);
constexpr size_t OFF_ERR = OFF_CURSOR + al256(sizeof(int) * NA_MAX_CAMS);
constexpr size_t NA_SCRATCH_BYTES = OFF_ERR + 256;   // about 10.9 MiB

// Host code must not use this name as an address: it is a host-side stand-in. The device
// address comes from cudaGetSymbolAddress (scratch_base below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 256;
std::mutex g_mu;
unsigned char *g_base[NA_MAX_DEVICES] = {};

cudaError_t scratch_base(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_base[dev];
    return cudaSuccess;
}

// ---- device-side checks of the caller's pair table -------------------------------------------
__global__ void k_na_check(const int *pair_off, const int *cam_i, const int *cam_j, int n_pairs,
                           int n_cams, int64_t n_pp, unsigned *err) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_pairs) return;
    bool ok = pair_off[n + 1] > pair_off[n];
    if (n == 0) ok = ok && pair_off[0] == 0;
    if (n == n_pairs - 1) ok = ok && (int64_t)pair_off[n_pairs] == n_pp;
    const int i = cam_i[n], j = cam_j[n];
    ok = ok && i >= 0 && i < n_cams && j >= 0 && j < n_cams && i != j;
    if (!ok) atomicOr(err, ERR_PAIR_RANGE);
}

// ---- camera -> (pair, role) lists, in pair order --------------------------------------------
// O(n_pairs) counting and filling with atomics, then every camera's list is put into pair order
// (the order in which the per-camera gradient sums are taken, so results are reproducible):
// each entry's rank is the number of smaller entries of the same camera, O(sum of squared
// camera degrees) in all.
__global__ void k_na_cam_count(const int *cam_i, const int *cam_j, int n_pairs, int *cnt) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_pairs) return;
    atomicAdd(&cnt[cam_i[n] + 1], 1);
    atomicAdd(&cnt[cam_j[n] + 1], 1);
}

__global__ void k_na_cam_scan(int *off, int n_cams) {  // one block: off[0] = 0, inclusive scan
    __shared__ int part[1024];
    const int per = (n_cams + 1023) / 1024;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int k = 0; k < per; ++k)
        if (b + k < n_cams) s += off[b + k + 1];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int x = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += x;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int k = 0; k < per; ++k)
        if (b + k < n_cams) {
            run += off[b + k + 1];
            off[b + k + 1] = run;
        }
    if (threadIdx.x == 0) off[0] = 0;
}

__global__ void k_na_cam_fill(const int *cam_i, const int *cam_j, int n_pairs, const int *off, int *cursor,
                              int *tmp) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_pairs) return;
    const int i = cam_i[n], j = cam_j[n];
    tmp[off[i] + atomicAdd(&cursor[i], 1)] = 2 * n;
    tmp[off[j] + atomicAdd(&cursor[j], 1)] = 2 * n + 1;
}

// one warp per camera: entry e goes to position off[k] + #{entries of k smaller than e}
__global__ void k_na_cam_order(const int *off, const int *tmp, int n_cams, int *ent) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= n_cams) return;
    const int b = off[k], e = off[k + 1];
    for (int a = b + lane; a < e; a += 32) {
        const int v = tmp[a];
        int rank = 0;
        for (int c = b; c < e; ++c) rank += tmp[c] < v ? 1 : 0;
        ent[b + rank] = v;
    }
}

// ---- streaming loss + adjoint with bounds-checked loads (caller buffers are not padded) ------
__device__ __forceinline__ void na_flush(float *slots, int seg, int r, int lane, float *acc) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        float v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[i] = v;
    }
    if (lane == 0) {
        float *s = slots + (size_t)(seg + r) * SLOT;
#pragma unroll
        for (int i = 0; i < 10; ++i) s[i] = acc[i];
    }
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = 0.f;
}

__global__ void __launch_bounds__(256) k_na_stream(DevProblem d, const float4 *kp, const float *w) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    const int64_t p_begin = (int64_t)r * WR;
    const int64_t p_end = min(p_begin + (int64_t)WR, d.n_pp);
    int seg = d.range_pair[r];
    int64_t seg_end = d.pair_off[seg + 1];
    float E[9], acc[10];
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = d.geo[(size_t)seg * GEO + k];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.f;
    const bool l1 = d.loss == FM_LOSS_L1;
    for (int64_t gb = p_begin; gb < p_end; gb += 32) {
        const int64_t q = gb + lane;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        float wq = 0.f;
        if (q < p_end) {
            v = kp[q];
            wq = w ? w[q] : 1.f;
            // the same input rules as fm_create_problem / fm_set_weights: finite coordinates
            // of magnitude <= 8, finite non-negative weights (the point pair is then skipped)
            const bool coord_ok = fabsf(v.x) <= COORD_LIMIT && fabsf(v.y) <= COORD_LIMIT &&
                                  fabsf(v.z) <= COORD_LIMIT && fabsf(v.w) <= COORD_LIMIT;
            const bool w_ok = wq >= 0.f && wq <= 3.0e38f;
            if (!coord_ok || !w_ok) {
                atomicOr(d.err, coord_ok ? ERR_WEIGHT : ERR_COORD);
                v = make_float4(0.f, 0.f, 0.f, 0.f);
                wq = 0.f;
            }
        }
        int64_t lo = gb;
        const int64_t g_end = min(gb + 32, p_end);
        while (true) {
            const int64_t hi = min(seg_end, p_end);
            if (q >= lo && q < hi) {
                const float r0 = fmaf(E[0], v.x, fmaf(E[1], v.y, E[2]));
                const float r1 = fmaf(E[3], v.x, fmaf(E[4], v.y, E[5]));
                const float r2 = fmaf(E[6], v.x, fmaf(E[7], v.y, E[8]));
                const float e = fmaf(v.z, r0, fmaf(v.w, r1, r2));
                float s;
                if (l1) {
                    s = e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f);
                    acc[9] += fabsf(e);
                } else {
                    s = wq * e;
                    acc[9] = fmaf(s, e, acc[9]);
                }
                const float a = s * v.z, b = s * v.w;
                acc[0] = fmaf(a, v.x, acc[0]);
                acc[1] = fmaf(a, v.y, acc[1]);
                acc[2] += a;
                acc[3] = fmaf(b, v.x, acc[3]);
                acc[4] = fmaf(b, v.y, acc[4]);
                acc[5] += b;
                acc[6] = fmaf(s, v.x, acc[6]);
                acc[7] = fmaf(s, v.y, acc[7]);
                acc[8] += s;
            }
            if (seg_end >= g_end) break;
            na_flush(d.slots, seg, r, lane, acc);
            lo = seg_end;
            ++seg;
            seg_end = d.pair_off[seg + 1];
#pragma unroll
            for (int k = 0; k < 9; ++k) E[k] = d.geo[(size_t)seg * GEO + k];
        }
    }
    na_flush(d.slots, seg, r, lane, acc);
}

}  // namespace
}  // namespace fm

using namespace fm;

// the library-wide last-error string lives in fm_api.cu
void fm_internal_set_error(const char *msg);

namespace {
fm_status na_fail(fm_status s, const char *msg) {
    fm_internal_set_error(msg);
    return s;
}
}  // namespace

#define NA_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return na_fail(FM_ECUDA, cudaGetErrorString(e_));        \
    } while (0)

extern "C" FM_API fm_status fm_loss_grad_noalloc(int32_t n_cams, const double *d_R,
                                                 const double *d_c, int32_t n_pairs,
                                                 const int32_t *d_cam_i, const int32_t *d_cam_j,
                                                 const int32_t *d_pair_off, int64_t n_pp,
                                                 const float *d_kp, const float *d_w, int32_t loss,
                                                 double *d_loss, double *d_grad, void *stream) {
    if (n_cams < 2 || n_cams > NA_MAX_CAMS)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: n_cams must be in [2, 4096]");
    if (n_pairs < 1 || n_pairs > NA_MAX_PAIRS)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: n_pairs must be in [1, 32768]");
    if (n_pp < n_pairs || n_pp > NA_MAX_PP)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: n_pp must be in [n_pairs, 2^26]");
    if (!d_R || !d_c || !d_cam_i || !d_cam_j || !d_pair_off || !d_kp || !d_loss || !d_grad)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: only d_w may be NULL");
    if (reinterpret_cast<uintptr_t>(d_kp) % 16 != 0)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: d_kp must be 16-byte aligned");
    if (loss != FM_LOSS_IRLS && loss != FM_LOSS_L1)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: loss must be FM_LOSS_IRLS or FM_LOSS_L1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    NA_CUDA(scratch_base(&base));

    DevProblem d{};
    d.n_cams = n_cams;
    d.n_pairs = n_pairs;
    d.n_pp = n_pp;
    d.n_pad = n_pp;
    d.n_ranges = (int)((n_pp + WR - 1) / WR);
    d.storage = FM_STORE_FP32;
    d.loss = loss;
    d.delta = 1e-6;
    d.w_scale = 1.0f;
    d.R = const_cast<double *>(d_R);
    d.c = const_cast<double *>(d_c);
    d.cam_i = const_cast<int *>(d_cam_i);
    d.cam_j = const_cast<int *>(d_cam_j);
    d.pair_off = const_cast<int *>(d_pair_off);
    d.cam = reinterpret_cast<float *>(base + OFF_CAM);
    d.cen = reinterpret_cast<float2 *>(base + OFF_CEN);
    d.geo = reinterpret_cast<float *>(base + OFF_GEO);
    d.range_pair = reinterpret_cast<int *>(base + OFF_RANGE);
    d.slots = reinterpret_cast<float *>(base + OFF_SLOTS);
    d.pair_grad = reinterpret_cast<float *>(base + OFF_PG);
    d.cam_off = reinterpret_cast<int *>(base + OFF_CAMOFF);
    d.cam_ent = reinterpret_cast<int *>(base + OFF_CAMENT);
    d.err = reinterpret_cast<unsigned *>(base + OFF_ERR);
    d.grad = d_grad;
    d.loss_out = d_loss;

    // the array keeps the previous call's contents: clear what must start at zero
    NA_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), s));
    NA_CUDA(cudaMemsetAsync(d.cen, 0, sizeof(float2) * n_cams, s));
    k_na_check<<<(n_pairs + 255) / 256, 256, 0, s>>>(d.pair_off, d.cam_i, d.cam_j, n_pairs, n_cams,
                                                      n_pp, d.err);
    NA_CUDA(cudaGetLastError());
    unsigned err = 0;
    NA_CUDA(cudaMemcpyAsync(&err, d.err, sizeof err, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (err)
        return na_fail(FM_EINVAL, "fm_loss_grad_noalloc: pair_off must rise strictly from 0 to n_pp "
                                  "and camera indices must be valid with cam_i != cam_j");

    int *cam_tmp = reinterpret_cast<int *>(base + OFF_CAMTMP);
    int *cursor = reinterpret_cast<int *>(base + OFF_CURSOR);
    NA_CUDA(cudaMemsetAsync(d.cam_off, 0, sizeof(int) * (n_cams + 1), s));
    NA_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * n_cams, s));
    launch_cam_prep(d, s);
    launch_range_pairs(d.pair_off, n_pairs, d.n_ranges, d.range_pair, s);
    k_na_cam_count<<<(n_pairs + 255) / 256, 256, 0, s>>>(d.cam_i, d.cam_j, n_pairs, d.cam_off);
    k_na_cam_scan<<<1, 1024, 0, s>>>(d.cam_off, n_cams);
    k_na_cam_fill<<<(n_pairs + 255) / 256, 256, 0, s>>>(d.cam_i, d.cam_j, n_pairs, d.cam_off, cursor, cam_tmp);
    k_na_cam_order<<<(n_cams + 7) / 8, 256, 0, s>>>(d.cam_off, cam_tmp, n_cams, d.cam_ent);
    launch_pair_setup(d, s);
    k_na_stream<<<(d.n_ranges + 7) / 8, 256, 0, s>>>(d, reinterpret_cast<const float4 *>(d_kp),
                                                      loss == FM_LOSS_IRLS ? d_w : nullptr);
    launch_combine(d, s);
    launch_gather(d, false, s);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemcpyAsync(&err, d.err, sizeof err, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (err & (ERR_COORD | ERR_WEIGHT))
        return na_fail(FM_EINVAL, (err & ERR_COORD)
                                      ? "fm_loss_grad_noalloc: keypoint coordinates must be finite with magnitude <= 8"
                                      : "fm_loss_grad_noalloc: weights must be finite and >= 0");
    if (err & (ERR_DEGENERATE | ERR_NONFINITE))
        return na_fail(FM_EDEGENERATE, "fm_loss_grad_noalloc: zero-length relative translation or "
                                       "non-finite loss/gradient");
    return FM_OK;
}
