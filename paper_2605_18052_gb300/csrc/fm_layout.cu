// One-off device layout of a problem: validation, stable sort by image pair, CSR offsets,
// warp-range table, per-image centroids and packing into the streaming format.
//
// The paper's point-pair sets Q_n (Sec. "Epipolar Adjustment") arrive as one flat list with a
// pair index per point pair; the streaming kernels want them contiguous per pair, so the
// layout sorts them (stable, so point pairs of one pair keep their input order and every
// reduction stays deterministic).
#include <algorithm>
#include <vector>

#include "fm_internal.cuh"

namespace fm {

static inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ---- validation ---------------------------------------------------------------------------------
__global__ void k_validate(const int *pair_id, const float2 *x1, const float2 *x2, int64_t n,
                           int n_pairs, unsigned *err) {
    unsigned bits = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int k = pair_id[p];
        if (k < 0 || k >= n_pairs) bits |= ERR_PAIR_RANGE;
        if (p > 0 && pair_id[p - 1] > k) bits |= ERR_UNSORTED;
        const float2 a = x1[p], b = x2[p];
        const bool ok = fabsf(a.x) <= COORD_LIMIT && fabsf(a.y) <= COORD_LIMIT &&
                        fabsf(b.x) <= COORD_LIMIT && fabsf(b.y) <= COORD_LIMIT;  // false for NaN
        if (!ok) bits |= ERR_COORD;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(err, bits);
}

void launch_validate(const int *pair_id, const float2 *x1, const float2 *x2, int64_t n_pp,
                     int n_pairs, unsigned *err, cudaStream_t s) {
    const int grid = std::min<int64_t>(blocks_for(n_pp, 256), 152 * 16);
    k_validate<<<grid, 256, 0, s>>>(pair_id, x1, x2, n_pp, n_pairs, err);
}

// ---- stable LSD radix sort of (pair id, input index) ----------------------------------------------
constexpr int SORT_THREADS = 256;
constexpr int SORT_TILE = 4096;
constexpr int RADIX = 256;

__global__ void __launch_bounds__(SORT_THREADS)
k_radix_hist(const int *keys, int64_t n, int shift, int n_tiles, unsigned *hist) {
    __shared__ unsigned h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int i = threadIdx.x; i < SORT_TILE; i += SORT_THREADS) {
        const int64_t p = base + i;
        if (p < n) atomicAdd(&h[(keys[p] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Scatter one tile; elements keep their input order within each digit (stable).
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_scatter(const int *keys_in, const int *vals_in, int64_t n, int shift, int n_tiles,
                const unsigned *offs, int *keys_out, int *vals_out) {
    __shared__ unsigned run[RADIX];
    __shared__ unsigned wcnt[SORT_THREADS / 32][RADIX];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    run[t] = offs[(size_t)t * n_tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int c = 0; c < SORT_TILE; c += SORT_THREADS) {
#pragma unroll
        for (int w = 0; w < SORT_THREADS / 32; ++w) wcnt[w][t] = 0;
        __syncthreads();
        const int64_t p = base + c + t;
        const bool valid = p < n;
        const int key = valid ? keys_in[p] : 0;
        const int val = valid ? (vals_in ? vals_in[p] : (int)p) : 0;
        const unsigned dig = valid ? (unsigned)((key >> shift) & (RADIX - 1)) : (unsigned)(RADIX + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const unsigned rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pos = run[dig] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][dig];
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        unsigned add = 0;
#pragma unroll
        for (int w = 0; w < SORT_THREADS / 32; ++w) add += wcnt[w][t];
        run[t] += add;
        __syncthreads();
    }
}

// exclusive scan (uint32), three levels of 1024-element blocks
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_BLOCK = 1024;

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_block(unsigned *data, int64_t n, unsigned *block_sums) {
    __shared__ unsigned s[SCAN_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + threadIdx.x * 4;
    unsigned v[4], tot = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? data[base + k] : 0u;
        tot += v[k];
    }
    s[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < SCAN_THREADS; o <<= 1) {  // Hillis-Steele inclusive scan
        const unsigned x = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned run = s[threadIdx.x] - tot;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1 && block_sums) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(unsigned *data, int64_t n, const unsigned *block_offsets) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) data[p] += block_offsets[p / SCAN_PER_BLOCK];
}

static void exclusive_scan(unsigned *data, int64_t n, unsigned *tmp, cudaStream_t s) {
    const int64_t nb = (n + SCAN_PER_BLOCK - 1) / SCAN_PER_BLOCK;
    if (nb <= 1) {
        k_scan_block<<<1, SCAN_THREADS, 0, s>>>(data, n, nullptr);
        return;
    }
    k_scan_block<<<(int)nb, SCAN_THREADS, 0, s>>>(data, n, tmp);
    exclusive_scan(tmp, nb, tmp + nb, s);
    k_scan_add<<<blocks_for(n, 256), 256, 0, s>>>(data, n, tmp);
}

cudaError_t sort_by_pair(const int *pair_id, int64_t n_pp, int n_pairs, int *keys_out,
                         int *perm_out, cudaStream_t s) {
    int bits = 0;
    while ((1ll << bits) < n_pairs) ++bits;
    const int passes = std::max(1, (bits + 7) / 8);
    const int n_tiles = (int)((n_pp + SORT_TILE - 1) / SORT_TILE);
    const int64_t hist_n = (int64_t)RADIX * n_tiles;
    int *kbuf = nullptr, *vbuf = nullptr;
    unsigned *hist = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(&kbuf, sizeof(int) * n_pp, s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync(&vbuf, sizeof(int) * n_pp, s)) != cudaSuccess) return e;
    // histogram + scan temporaries (scan levels need < hist_n / 512 extra entries)
    if ((e = cudaMallocAsync(&hist, sizeof(unsigned) * (hist_n + hist_n / 512 + 64), s)) != cudaSuccess)
        return e;
    // ping-pong so that the last pass lands in (keys_out, perm_out)
    const int *kin = pair_id;
    const int *vin = nullptr;
    for (int pass = 0; pass < passes; ++pass) {
        const bool to_out = ((passes - 1 - pass) % 2) == 0;
        int *kout = to_out ? keys_out : kbuf;
        int *vout = to_out ? perm_out : vbuf;
        k_radix_hist<<<n_tiles, SORT_THREADS, 0, s>>>(kin, n_pp, 8 * pass, n_tiles, hist);
        exclusive_scan(hist, hist_n, hist + hist_n, s);
        k_radix_scatter<<<n_tiles, SORT_THREADS, 0, s>>>(kin, vin, n_pp, 8 * pass, n_tiles, hist,
                                                         kout, vout);
        kin = kout;
        vin = vout;
    }
    cudaFreeAsync(kbuf, s);
    cudaFreeAsync(vbuf, s);
    cudaFreeAsync(hist, s);
    return cudaGetLastError();
}

// ---- CSR offsets from sorted pair ids -----------------------------------------------------------------
__global__ void k_pair_starts(const int *keys, int64_t n, int *pair_off) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int k = keys[p];
    if (p == 0 || keys[p - 1] != k) pair_off[k] = (int)p;
}

__global__ void k_pair_check(int *pair_off, int n_pairs, int64_t n_pp, unsigned *err) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < n_pairs && pair_off[n] < 0) atomicOr(err, ERR_EMPTY_PAIR);
    if (n == n_pairs) pair_off[n] = (int)n_pp;
}

void launch_pair_offsets(const int *sorted_keys, int64_t n_pp, int n_pairs, int *pair_off,
                         unsigned *err, cudaStream_t s) {
    cudaMemsetAsync(pair_off, 0xff, sizeof(int) * (n_pairs + 1), s);
    k_pair_starts<<<blocks_for(n_pp, 256), 256, 0, s>>>(sorted_keys, n_pp, pair_off);
    k_pair_check<<<blocks_for(n_pairs + 1, 256), 256, 0, s>>>(pair_off, n_pairs, n_pp, err);
}

// first pair of every warp range: the largest n with pair_off[n] <= r * WR
__global__ void k_range_pairs(const int *pair_off, int n_pairs, int n_ranges, int *range_pair) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_ranges) return;
    const long long p = (long long)r * WR;
    int lo = 0, hi = n_pairs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pair_off[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    range_pair[r] = lo;
}

void launch_range_pairs(const int *pair_off, int n_pairs, int n_ranges, int *range_pair,
                        cudaStream_t s) {
    k_range_pairs<<<blocks_for(n_ranges, 256), 256, 0, s>>>(pair_off, n_pairs, n_ranges, range_pair);
}

// ---- per-image centroids (FP16 storage) ---------------------------------------------------------------
// c_k = mean of every keypoint of image k over all its pairs, summed exactly as trunc(x * 2^32)
// in int64 (order-independent), then (double)sum / count * 2^-32 rounded to FP32.
// Warp r walks the sorted point pairs of warp range r (as the streaming kernels do) and keeps
// the four fixed-point sums of the current image pair in registers; when the pair ends the
// warp reduces them and lane 0 adds them to the pair's two cameras (one atomic set per
// (range, pair) intersection, integer adds, so the result does not depend on their order).
__device__ __forceinline__ void centroid_flush(const DevProblem &d, int seg, int lane,
                                               long long *f, unsigned long long *sums) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
    if (lane == 0) {
        const int i = d.cam_i[seg], j = d.cam_j[seg];
        atomicAdd(&sums[2 * i], (unsigned long long)f[0]);
        atomicAdd(&sums[2 * i + 1], (unsigned long long)f[1]);
        atomicAdd(&sums[2 * j], (unsigned long long)f[2]);
        atomicAdd(&sums[2 * j + 1], (unsigned long long)f[3]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = 0;
}

__global__ void k_centroid_sums(DevProblem d, const float2 *x1, const float2 *x2,
                                unsigned long long *sums) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= d.n_ranges) return;
    const int64_t p_begin = (int64_t)r * WR;
    const int64_t p_end = min(p_begin + (int64_t)WR, d.n_pp);
    int seg = d.range_pair[r];
    int64_t seg_end = d.pair_off[seg + 1];
    long long f[4] = {0, 0, 0, 0};
    const float sc = 4294967296.0f;  // 2^FIXED_SHIFT
    for (int64_t gb = p_begin; gb < p_end; gb += 32) {
        const int64_t q = gb + lane;
        long long v[4] = {0, 0, 0, 0};
        if (q < p_end) {
            const int64_t src = d.perm ? d.perm[q] : q;
            const float2 a = x1[src], b = x2[src];
            v[0] = __float2ll_rz(a.x * sc);
            v[1] = __float2ll_rz(a.y * sc);
            v[2] = __float2ll_rz(b.x * sc);
            v[3] = __float2ll_rz(b.y * sc);
        }
        int64_t lo = gb;
        const int64_t g_end = min(gb + 32, p_end);
        while (true) {
            const int64_t hi = min(seg_end, p_end);
            if (q >= lo && q < hi) {
#pragma unroll
                for (int k = 0; k < 4; ++k) f[k] += v[k];
            }
            if (seg_end >= g_end) break;
            centroid_flush(d, seg, lane, f, sums);
            lo = seg_end;
            ++seg;
            seg_end = d.pair_off[seg + 1];
        }
    }
    centroid_flush(d, seg, lane, f, sums);
}

__global__ void k_centroid_final(const unsigned long long *sums, const int *cam_off,
                                 const int *cam_ent, const int *pair_off, int n_cams, float2 *cen) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_cams) return;
    long long cnt = 0;
    for (int e = cam_off[k]; e < cam_off[k + 1]; ++e) {
        const int n = cam_ent[e] >> 1;
        cnt += pair_off[n + 1] - pair_off[n];
    }
    float2 c = make_float2(0.f, 0.f);
    if (cnt > 0) {
        const double inv_scale = 1.0 / 4294967296.0;
        const double den = (double)cnt;
        c.x = __double2float_rn(__ddiv_rn(__ll2double_rn((long long)sums[2 * k]), den) * inv_scale);
        c.y = __double2float_rn(__ddiv_rn(__ll2double_rn((long long)sums[2 * k + 1]), den) * inv_scale);
    }
    cen[k] = c;
}

void launch_centroids(const DevProblem &d, const int *sorted_keys, const float2 *x1,
                      const float2 *x2, unsigned long long *sums, cudaStream_t s) {
    (void)sorted_keys;  // the walk uses pair_off and range_pair instead
    cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * 2 * d.n_cams, s);
    k_centroid_sums<<<blocks_for(d.n_ranges, 8), 256, 0, s>>>(d, x1, x2, sums);
    k_centroid_final<<<blocks_for(d.n_cams, 128), 128, 0, s>>>(sums, d.cam_off, d.cam_ent,
                                                              d.pair_off, d.n_cams, d.cen);
}

// ---- packing into the streaming format ------------------------------------------------------------
__global__ void k_pack(DevProblem d, const int *keys, const float2 *x1, const float2 *x2) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n_pad) return;
    if (d.storage == FM_STORE_FP32) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < d.n_pp) {
            const int64_t src = d.perm ? d.perm[p] : p;
            const float2 a = x1[src], b = x2[src];
            v = make_float4(a.x, a.y, b.x, b.y);
        }
        static_cast<float4 *>(d.kp)[p] = v;
    } else {
        uint2 v = make_uint2(0u, 0u);
        if (p < d.n_pp) {
            const int64_t src = d.perm ? d.perm[p] : p;
            const int n = keys[p];
            const float2 a = x1[src], b = x2[src];
            const float2 ci = d.cen[d.cam_i[n]], cj = d.cen[d.cam_j[n]];
            // offsets: FP32 difference, then round to nearest FP16
            const __half2 h1 = __halves2half2(__float2half_rn(__fsub_rn(a.x, ci.x)),
                                              __float2half_rn(__fsub_rn(a.y, ci.y)));
            const __half2 h2 = __halves2half2(__float2half_rn(__fsub_rn(b.x, cj.x)),
                                              __float2half_rn(__fsub_rn(b.y, cj.y)));
            v.x = *reinterpret_cast<const unsigned *>(&h1);
            v.y = *reinterpret_cast<const unsigned *>(&h2);
        }
        static_cast<uint2 *>(d.kp)[p] = v;
    }
}

void launch_pack(const DevProblem &d, const int *sorted_keys, const float2 *x1, const float2 *x2,
                 cudaStream_t s) {
    k_pack<<<blocks_for(d.n_pad, 256), 256, 0, s>>>(d, sorted_keys, x1, x2);
}

// ---- weights ------------------------------------------------------------------------------------------
__device__ __forceinline__ void store_weight(const DevProblem &d, int64_t p, float w) {
    if (d.storage == FM_STORE_FP32) static_cast<float *>(d.w)[p] = w;
    else static_cast<__half *>(d.w)[p] = __float2half_rn(w * d.w_scale);
}

__device__ __forceinline__ float read_weight(const DevProblem &d, int64_t p) {
    if (d.storage == FM_STORE_FP32) return static_cast<const float *>(d.w)[p];
    return __half2float(static_cast<const __half *>(d.w)[p]) / d.w_scale;
}

__global__ void k_fill_weights(DevProblem d, float value) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < d.n_pad) store_weight(d, p, p < d.n_pp ? value : 0.f);
}

void launch_fill_weights(const DevProblem &d, float value, cudaStream_t s) {
    k_fill_weights<<<blocks_for(d.n_pad, 256), 256, 0, s>>>(d, value);
}

__global__ void k_set_weights(DevProblem d, const float *w_in) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n_pp) return;
    const float w = w_in[d.perm ? d.perm[p] : p];
    const bool ok = w >= 0.f && w <= (float)(1.0 / d.delta);  // false for NaN
    if (!ok) atomicOr(d.err, ERR_WEIGHT);
    store_weight(d, p, ok ? w : 0.f);
}

void launch_set_weights(const DevProblem &d, const float *w_input_order, cudaStream_t s) {
    k_set_weights<<<blocks_for(d.n_pp, 256), 256, 0, s>>>(d, w_input_order);
}

__global__ void k_get_weights(DevProblem d, float *w_out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n_pp) return;
    w_out[d.perm ? d.perm[p] : p] = read_weight(d, p);
}

void launch_get_weights(const DevProblem &d, float *w_input_order, cudaStream_t s) {
    k_get_weights<<<blocks_for(d.n_pp, 256), 256, 0, s>>>(d, w_input_order);
}

__global__ void k_unpermute(const int *perm, int64_t n, const float *sorted, float *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[perm ? perm[p] : p] = sorted[p];
}

void launch_unpermute(const DevProblem &d, const float *sorted, float *input_order,
                      cudaStream_t s) {
    k_unpermute<<<blocks_for(d.n_pp, 256), 256, 0, s>>>(d.perm, d.n_pp, sorted, input_order);
}

__global__ void k_fill_half(__half *p, int64_t n, float value) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) p[q] = __float2half_rn(value);
}

void launch_fill_half(__half *p, int64_t n, float value, cudaStream_t s) {
    k_fill_half<<<blocks_for(n, 256), 256, 0, s>>>(p, n, value);
}

__global__ void k_set_scores(DevProblem d, const float *score_in) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= d.n_pp) return;
    const float v = score_in[d.perm ? d.perm[q] : q];
    const bool ok = v >= 0.f && v <= 1.f;  // false for NaN
    if (!ok) atomicOr(d.err, ERR_WEIGHT);
    d.score[q] = __float2half_rn(ok ? v : 0.5f);
}

void launch_set_scores(const DevProblem &d, const float *score_input_order, cudaStream_t s) {
    k_set_scores<<<blocks_for(d.n_pp, 256), 256, 0, s>>>(d, score_input_order);
}

}  // namespace fm
