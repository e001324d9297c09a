// Global translation stage (Sec. "Global Translation", Eq. fastmap-global-translation-objective):
// camera centres o_k from unit relative translations with the rotations fixed,
//   L_t = (1/|P|) sum_n || (o_j - o_i)/||o_j - o_i|| - o_{i->j} ||_1,   o_{i->j} = -R_j^T t_{i->j},
// by Adam from random initial centres, several runs at once, and the merge of the runs
// (centre, unit mean norm, per camera the run with the lowest mean pair loss).
//
// Per iteration two launches, chained with programmatic dependent launch:
//   k_tr_pair  (pair, run)   : the pair's L1 term and its subgradient with respect to
//                              u = o_j - o_i, projected orthogonally to u and divided by |u|
//   k_tr_cam   (camera, run) : the camera's gradient gathered from its pairs (CSR of the pair
//                              table, fixed order, no atomics), its mean pair loss, Adam
// then one launch closes a chain (per-run loss total, step count). Centres and their update
// are FP64; the per-pair arithmetic is FP32 on the FP64 difference o_j - o_i.
#include <cmath>
#include <string>
#include <vector>

#include "fm_walk.cuh"

void fm_internal_set_error(const char *msg);

using namespace fm;

namespace {

constexpr int TR_THREADS = 256;
constexpr int TR_CAMS = 8;   // cameras (warps) per block of the camera kernel

struct DevTrans {
    int n_cams, n_pairs, n_runs;
    const int *cam_i, *cam_j, *cam_off, *cam_ent;
    float4 *oij;             // per pair: o_{i->j} (xyz), 0
    double *o;               // n_runs x n_cams x 3
    float *m, *v;            // Adam moments, same shape
    float4 *pterm;           // n_runs x n_pairs: gradient wrt u (xyz), L1 term
    float *cam_loss;         // n_runs x n_cams: mean L1 term of the camera's pairs
    double *grad;            // n_runs x n_cams x 3 (gradient-only evaluation)
    double *blk_loss;        // n_runs x camera-kernel blocks
    double *loss;            // n_runs
    double *stats;           // n_runs x 4: mean (3), mean norm after centring
    double *hyper;           // lr, beta1, beta2, eps
    long long *step;
    unsigned *err;
};

__host__ __device__ inline int cam_blocks(const DevTrans &t) { return (t.n_cams + TR_CAMS - 1) / TR_CAMS; }

__global__ void k_tr_setup(DevTrans t, const double *R, const double *trel) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= t.n_pairs) return;
    const double *Rj = R + (size_t)t.cam_j[n] * 9;
    const double *tn = trel + (size_t)n * 3;
    double o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = -(Rj[a] * tn[0] + Rj[3 + a] * tn[1] + Rj[6 + a] * tn[2]);
    t.oij[n] = make_float4((float)o[0], (float)o[1], (float)o[2], 0.f);
}

__device__ __forceinline__ float sgn(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(TR_THREADS) k_tr_pair(DevTrans t) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int run = blockIdx.y;
    const int i = n < t.n_pairs ? t.cam_i[n] : 0, j = n < t.n_pairs ? t.cam_j[n] : 0;
    const float4 target = n < t.n_pairs ? t.oij[n] : make_float4(0.f, 0.f, 0.f, 0.f);
    pdl_wait();     // centres of the previous step
    pdl_trigger();
    if (n >= t.n_pairs) return;
    const double *oi = t.o + ((size_t)run * t.n_cams + i) * 3;
    const double *oj = t.o + ((size_t)run * t.n_cams + j) * 3;
    const float u[3] = {(float)(oj[0] - oi[0]), (float)(oj[1] - oi[1]), (float)(oj[2] - oi[2])};
    const float n2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(n2 > 0.f) || !isfinite(n2)) {
        atomicOr(t.err, ERR_DEGENERATE);
        t.pterm[(size_t)run * t.n_pairs + n] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float nrm = sqrtf(n2);
    const float uh[3] = {u[0] / nrm, u[1] / nrm, u[2] / nrm};
    const float r[3] = {uh[0] - target.x, uh[1] - target.y, uh[2] - target.z};
    const float term = fabsf(r[0]) + fabsf(r[1]) + fabsf(r[2]);
    const float s[3] = {sgn(r[0]), sgn(r[1]), sgn(r[2])};
    const float dot = uh[0] * s[0] + uh[1] * s[1] + uh[2] * s[2];
    t.pterm[(size_t)run * t.n_pairs + n] =
        make_float4((s[0] - uh[0] * dot) / nrm, (s[1] - uh[1] * dot) / nrm, (s[2] - uh[2] * dot) / nrm, term);
}

// warp per camera; apply = 0 writes the gradient instead of stepping
__global__ void __launch_bounds__(TR_CAMS * 32) k_tr_cam(DevTrans t, int it, int apply) {
    __shared__ double s_loss[TR_CAMS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int run = blockIdx.y;
    const int k = blockIdx.x * TR_CAMS + warp;
    const int e_begin = k < t.n_cams ? t.cam_off[k] : 0;
    const int e_end = k < t.n_cams ? t.cam_off[k + 1] : 0;
    pdl_wait();     // pair terms of this step
    pdl_trigger();
    float g[3] = {0.f, 0.f, 0.f}, tsum = 0.f, lsum = 0.f;
    for (int e = e_begin + lane; e < e_end; e += 32) {
        const int ent = t.cam_ent[e];
        const int n = ent >> 1, role = ent & 1;
        const float4 p = t.pterm[(size_t)run * t.n_pairs + n];
        const float sg = role ? 1.f : -1.f;   // camera j: +dL/du, camera i: -dL/du
        g[0] = fmaf(sg, p.x, g[0]);
        g[1] = fmaf(sg, p.y, g[1]);
        g[2] = fmaf(sg, p.z, g[2]);
        tsum += p.w;
        if (role == 0) lsum += p.w;          // each pair's loss counted once
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) g[a] += __shfl_xor_sync(0xffffffffu, g[a], o);
        tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if (lane == 0) {
        s_loss[warp] = (double)lsum;
        if (k < t.n_cams) {
            const size_t base = ((size_t)run * t.n_cams + k) * 3;
            const int cnt = e_end - e_begin;
            t.cam_loss[(size_t)run * t.n_cams + k] = cnt > 0 ? tsum / (float)cnt : 0.f;
            const double inv_b = 1.0 / (double)t.n_pairs;
            if (!apply) {
#pragma unroll
                for (int a = 0; a < 3; ++a) t.grad[base + a] = (double)g[a] * inv_b;
            } else {
                const long long ts = *t.step + 1 + it;
                const float lr = (float)t.hyper[0], b1 = (float)t.hyper[1], b2 = (float)t.hyper[2],
                            eps = (float)t.hyper[3];
                const float bc1 = 1.f - powf(b1, (float)ts), bc2 = 1.f - powf(b2, (float)ts);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float ga = (float)((double)g[a] * inv_b);
                    const float mo = b1 * t.m[base + a] + (1.f - b1) * ga;
                    const float vo = b2 * t.v[base + a] + (1.f - b2) * ga * ga;
                    t.m[base + a] = mo;
                    t.v[base + a] = vo;
                    t.o[base + a] -= (double)(lr * (mo / bc1) / (sqrtf(vo / bc2) + eps));
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
#pragma unroll
        for (int w = 0; w < TR_CAMS; ++w) b += s_loss[w];
        t.blk_loss[(size_t)run * cam_blocks(t) + blockIdx.x] = b;
    }
}

// per run: loss total (FP64, fixed order) / |P|; block 0 adds `count` to the step count
__global__ void __launch_bounds__(TR_THREADS) k_tr_finalize(DevTrans t, int count) {
    __shared__ double red[TR_THREADS];
    pdl_wait();
    pdl_trigger();
    const int run = blockIdx.x, nb = cam_blocks(t);
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += TR_THREADS) s += t.blk_loss[(size_t)run * nb + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = TR_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        t.loss[run] = red[0] / (double)t.n_pairs;
        if (run == 0) *t.step += count;
    }
}

// per run: centroid, then mean distance to it (FP64, fixed order)
__global__ void __launch_bounds__(TR_THREADS) k_tr_stats(DevTrans t) {
    __shared__ double red[4][TR_THREADS];
    const int run = blockIdx.x;
    const double *o = t.o + (size_t)run * t.n_cams * 3;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < t.n_cams; k += TR_THREADS)
        for (int a = 0; a < 3; ++a) s[a] += o[(size_t)k * 3 + a];
    for (int a = 0; a < 3; ++a) red[a][threadIdx.x] = s[a];
    __syncthreads();
    for (int w = TR_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int a = 0; a < 3; ++a) red[a][threadIdx.x] += red[a][threadIdx.x + w];
        __syncthreads();
    }
    const double mean[3] = {red[0][0] / t.n_cams, red[1][0] / t.n_cams, red[2][0] / t.n_cams};
    __syncthreads();
    double nsum = 0.0;
    for (int k = threadIdx.x; k < t.n_cams; k += TR_THREADS) {
        const double dx = o[(size_t)k * 3] - mean[0], dy = o[(size_t)k * 3 + 1] - mean[1],
                     dz = o[(size_t)k * 3 + 2] - mean[2];
        nsum += sqrt(dx * dx + dy * dy + dz * dz);
    }
    red[3][threadIdx.x] = nsum;
    __syncthreads();
    for (int w = TR_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[3][threadIdx.x] += red[3][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) t.stats[run * 4 + a] = mean[a];
        t.stats[run * 4 + 3] = red[3][0] / t.n_cams;
    }
}

// per camera: the normalised centre of the run with the lowest camera loss (first on ties),
// written to run 0
__global__ void k_tr_merge(DevTrans t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_cams) return;
    int best = 0;
    float bl = t.cam_loss[k];
    for (int r = 1; r < t.n_runs; ++r) {
        const float l = t.cam_loss[(size_t)r * t.n_cams + k];
        if (l < bl) {
            bl = l;
            best = r;
        }
    }
    const double *st = t.stats + best * 4;
    const double *src = t.o + ((size_t)best * t.n_cams + k) * 3;
    const double val[3] = {(src[0] - st[0]) / st[3], (src[1] - st[1]) / st[3], (src[2] - st[2]) / st[3]};
    for (int a = 0; a < 3; ++a) t.o[(size_t)k * 3 + a] = val[a];
}

}  // namespace

struct fm_translation {
    DevTrans d{};
    fm_translation_options opt{};
    int runs_total = 0;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr, graph8 = nullptr;
    std::vector<void *> allocs;
};

namespace {

fm_status tfail(fm_status s, const std::string &msg) {
    fm_internal_set_error(msg.c_str());
    return s;
}

#define TR_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return tfail(e_ == cudaErrorMemoryAllocation ? FM_ENOMEM : FM_ECUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

template <class T>
cudaError_t talloc(fm_translation *p, T **ptr, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) p->allocs.push_back(*ptr);
    return e;
}

cudaError_t tjoin_in(fm_translation *p) {
    cudaError_t e = cudaEventRecord(p->ev_in, p->user);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->s, p->ev_in, 0);
}

cudaError_t tjoin_out(fm_translation *p) {
    cudaError_t e = cudaEventRecord(p->ev_out, p->s);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->user, p->ev_out, 0);
}

fm_status tcheck_errors(fm_translation *p) {
    unsigned err = 0;
    TR_CUDA(cudaMemcpyAsync(&err, p->d.err, sizeof err, cudaMemcpyDeviceToHost, p->s));
    TR_CUDA(cudaStreamSynchronize(p->s));
    if (err & ERR_DEGENERATE) {
        const unsigned zero = 0;
        TR_CUDA(cudaMemcpyAsync(p->d.err, &zero, sizeof zero, cudaMemcpyHostToDevice, p->s));
        TR_CUDA(cudaStreamSynchronize(p->s));
        return tfail(FM_EDEGENERATE, "two cameras of an image pair share a centre or a centre is not finite");
    }
    return FM_OK;
}

void enqueue_eval(fm_translation *p, int it, bool apply, bool pdl) {
    const dim3 gp((p->d.n_pairs + TR_THREADS - 1) / TR_THREADS, p->d.n_runs);
    const dim3 gc(cam_blocks(p->d), p->d.n_runs);
    launch_k(k_tr_pair, gp, dim3(TR_THREADS), p->s, pdl, p->d);
    launch_k(k_tr_cam, gc, dim3(TR_CAMS * 32), p->s, true, p->d, it, apply ? 1 : 0);
}

void enqueue_steps(fm_translation *p, int iters) {
    for (int it = 0; it < iters; ++it) enqueue_eval(p, it, true, true);
    launch_k(k_tr_finalize, dim3(p->d.n_runs), dim3(TR_THREADS), p->s, true, p->d, iters);
}

fm_status build_tgraph(fm_translation *p, int iters, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    TR_CUDA(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
    enqueue_steps(p, iters);
    cudaError_t e = cudaStreamEndCapture(p->s, &g);
    if (e != cudaSuccess) return tfail(FM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return tfail(FM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return FM_OK;
}

void drop_graphs(fm_translation *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->graph8) cudaGraphExecDestroy(p->graph8);
    p->graph = p->graph8 = nullptr;
}

void free_trans(fm_translation *p) {
    if (!p) return;
    if (p->s) cudaStreamSynchronize(p->s);
    for (void *a : p->allocs) cudaFree(a);
    drop_graphs(p);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
}

bool finite_all(const double *a, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

fm_status tcheck(const fm_translation *p) {
    if (!p) return tfail(FM_EINVAL, "translation problem is NULL");
    return FM_OK;
}

fm_status upload_hyper(fm_translation *p) {
    const double h[4] = {p->opt.lr, p->opt.beta1, p->opt.beta2, p->opt.adam_eps};
    TR_CUDA(cudaMemcpyAsync(p->d.hyper, h, sizeof h, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

fm_status create_trans(fm_translation *p, int32_t n_cams, const double *R, int32_t n_pairs, const int32_t *cam_i,
                       const int32_t *cam_j, const double *t_rel, int32_t n_runs, const double *o_init) {
    DevTrans &d = p->d;
    d.n_cams = n_cams;
    d.n_pairs = n_pairs;
    d.n_runs = n_runs;
    p->runs_total = n_runs;
    TR_CUDA(cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking));
    TR_CUDA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
    TR_CUDA(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    TR_CUDA(tjoin_in(p));
    std::vector<int> cam_off(n_cams + 1, 0), cam_ent(2 * (size_t)n_pairs);
    for (int n = 0; n < n_pairs; ++n) {
        cam_off[cam_i[n] + 1]++;
        cam_off[cam_j[n] + 1]++;
    }
    for (int k = 0; k < n_cams; ++k) cam_off[k + 1] += cam_off[k];
    {
        std::vector<int> fill(cam_off.begin(), cam_off.end() - 1);
        for (int n = 0; n < n_pairs; ++n) {
            cam_ent[fill[cam_i[n]]++] = 2 * n;
            cam_ent[fill[cam_j[n]]++] = 2 * n + 1;
        }
    }
    const size_t nc3 = (size_t)n_runs * n_cams * 3;
    int *ci = nullptr, *cj = nullptr, *co = nullptr, *ce = nullptr;
    double *Rd = nullptr, *td = nullptr;
    TR_CUDA(talloc(p, &ci, (size_t)n_pairs));
    TR_CUDA(talloc(p, &cj, (size_t)n_pairs));
    TR_CUDA(talloc(p, &co, (size_t)n_cams + 1));
    TR_CUDA(talloc(p, &ce, 2 * (size_t)n_pairs));
    d.cam_i = ci;
    d.cam_j = cj;
    d.cam_off = co;
    d.cam_ent = ce;
    TR_CUDA(talloc(p, &d.oij, (size_t)n_pairs));
    TR_CUDA(talloc(p, &d.o, nc3));
    TR_CUDA(talloc(p, &d.m, nc3));
    TR_CUDA(talloc(p, &d.v, nc3));
    TR_CUDA(talloc(p, &d.pterm, (size_t)n_runs * n_pairs));
    TR_CUDA(talloc(p, &d.cam_loss, (size_t)n_runs * n_cams));
    TR_CUDA(talloc(p, &d.grad, nc3));
    TR_CUDA(talloc(p, &d.blk_loss, (size_t)n_runs * cam_blocks(d)));
    TR_CUDA(talloc(p, &d.loss, (size_t)n_runs));
    TR_CUDA(talloc(p, &d.stats, 4 * (size_t)n_runs));
    TR_CUDA(talloc(p, &d.hyper, 4));
    TR_CUDA(talloc(p, &d.step, 1));
    TR_CUDA(talloc(p, &d.err, 1));
    TR_CUDA(cudaMallocAsync(&Rd, sizeof(double) * 9 * n_cams, p->s));
    TR_CUDA(cudaMallocAsync(&td, sizeof(double) * 3 * n_pairs, p->s));
    TR_CUDA(cudaMemcpyAsync(ci, cam_i, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(cj, cam_j, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(co, cam_off.data(), sizeof(int) * (n_cams + 1), cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(ce, cam_ent.data(), sizeof(int) * 2 * n_pairs, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(Rd, R, sizeof(double) * 9 * n_cams, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(td, t_rel, sizeof(double) * 3 * n_pairs, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemcpyAsync(d.o, o_init, sizeof(double) * nc3, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemsetAsync(d.m, 0, sizeof(float) * nc3, p->s));
    TR_CUDA(cudaMemsetAsync(d.v, 0, sizeof(float) * nc3, p->s));
    TR_CUDA(cudaMemsetAsync(d.step, 0, sizeof(long long), p->s));
    TR_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), p->s));
    k_tr_setup<<<(n_pairs + TR_THREADS - 1) / TR_THREADS, TR_THREADS, 0, p->s>>>(d, Rd, td);
    TR_CUDA(cudaGetLastError());
    TR_CUDA(cudaFreeAsync(Rd, p->s));
    TR_CUDA(cudaFreeAsync(td, p->s));
    if (fm_status st = upload_hyper(p)) return st;
    TR_CUDA(tjoin_out(p));
    return FM_OK;
}

}  // namespace

extern "C" {

FM_API void fm_translation_default_options(fm_translation_options *opt) {
    if (!opt) return;
    opt->lr = 1e-2;
    opt->beta1 = 0.9;
    opt->beta2 = 0.999;
    opt->adam_eps = 1e-12;
    opt->use_graph = 1;
    opt->reserved = 0;
}

FM_API fm_status fm_translation_create(int32_t n_cams, const double *R, int32_t n_pairs, const int32_t *cam_i,
                                       const int32_t *cam_j, const double *t_rel, int32_t n_runs,
                                       const double *o_init, const fm_translation_options *opt, void *stream,
                                       fm_translation **out) {
    if (!out) return tfail(FM_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n_cams < 2) return tfail(FM_EINVAL, "n_cams must be >= 2");
    if (n_pairs < 1) return tfail(FM_EINVAL, "n_pairs must be >= 1");
    if (n_runs < 1 || n_runs > 65535) return tfail(FM_EINVAL, "n_runs must be in [1, 65535]");
    if (!R || !cam_i || !cam_j || !t_rel || !o_init) return tfail(FM_EINVAL, "array arguments must not be NULL");
    for (int n = 0; n < n_pairs; ++n)
        if (cam_i[n] < 0 || cam_i[n] >= n_cams || cam_j[n] < 0 || cam_j[n] >= n_cams || cam_i[n] == cam_j[n])
            return tfail(FM_EINVAL, "camera indices must be in [0, n_cams) with cam_i != cam_j");
    if (!finite_all(R, 9 * (size_t)n_cams) || !finite_all(t_rel, 3 * (size_t)n_pairs) ||
        !finite_all(o_init, 3 * (size_t)n_cams * n_runs))
        return tfail(FM_EINVAL, "rotations, relative translations and initial centres must be finite");
    for (int n = 0; n < n_pairs; ++n) {
        const double *t = t_rel + 3 * (size_t)n;
        const double l = std::sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (std::fabs(l - 1.0) > 1e-6) return tfail(FM_EINVAL, "relative translations must have unit length");
    }
    fm_translation_options o;
    fm_translation_default_options(&o);
    if (opt) o = *opt;
    if (!(o.lr > 0.0) || !(o.beta1 >= 0.0 && o.beta1 < 1.0) || !(o.beta2 >= 0.0 && o.beta2 < 1.0) ||
        !(o.adam_eps > 0.0) || (o.use_graph != 0 && o.use_graph != 1))
        return tfail(FM_EINVAL, "invalid options");
    fm_translation *p = new (std::nothrow) fm_translation();
    if (!p) return tfail(FM_ENOMEM, "host allocation failed");
    p->opt = o;
    p->user = static_cast<cudaStream_t>(stream);
    fm_status st = create_trans(p, n_cams, R, n_pairs, cam_i, cam_j, t_rel, n_runs, o_init);
    if (st != FM_OK) {
        free_trans(p);
        return st;
    }
    *out = p;
    return FM_OK;
}

FM_API void fm_translation_destroy(fm_translation *p) { free_trans(p); }

FM_API int32_t fm_translation_num_runs(const fm_translation *p) { return p ? p->d.n_runs : 0; }

FM_API fm_status fm_translation_set_learning_rate(fm_translation *p, double lr) {
    if (fm_status st = tcheck(p)) return st;
    if (!(lr > 0.0) || std::isinf(lr)) return tfail(FM_EINVAL, "lr must be finite and > 0");
    TR_CUDA(tjoin_in(p));
    p->opt.lr = lr;
    return upload_hyper(p);
}

FM_API fm_status fm_translation_loss_grad(fm_translation *p, double *loss, double *grad, double *cam_loss) {
    if (fm_status st = tcheck(p)) return st;
    if (!loss) return tfail(FM_EINVAL, "loss must not be NULL");
    TR_CUDA(tjoin_in(p));
    enqueue_eval(p, 0, false, false);
    launch_k(k_tr_finalize, dim3(p->d.n_runs), dim3(TR_THREADS), p->s, true, p->d, 0);
    TR_CUDA(cudaGetLastError());
    const size_t nc = (size_t)p->d.n_runs * p->d.n_cams;
    TR_CUDA(cudaMemcpyAsync(loss, p->d.loss, sizeof(double) * p->d.n_runs, cudaMemcpyDeviceToHost, p->s));
    if (grad) TR_CUDA(cudaMemcpyAsync(grad, p->d.grad, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, p->s));
    std::vector<float> cl;
    if (cam_loss) {
        cl.resize(nc);
        TR_CUDA(cudaMemcpyAsync(cl.data(), p->d.cam_loss, sizeof(float) * nc, cudaMemcpyDeviceToHost, p->s));
    }
    if (fm_status st = tcheck_errors(p)) return st;
    for (size_t i = 0; i < cl.size(); ++i) cam_loss[i] = cl[i];
    return FM_OK;
}

FM_API fm_status fm_translation_step(fm_translation *p, int32_t n_iters) {
    if (fm_status st = tcheck(p)) return st;
    if (n_iters < 0) return tfail(FM_EINVAL, "n_iters must be >= 0");
    if (n_iters == 0) return FM_OK;
    TR_CUDA(tjoin_in(p));
    if (!p->opt.use_graph) {
        enqueue_steps(p, n_iters);
        TR_CUDA(cudaGetLastError());
    } else {
        if (!p->graph)
            if (fm_status st = build_tgraph(p, 1, &p->graph)) return st;
        if (n_iters >= 8 && !p->graph8)
            if (fm_status st = build_tgraph(p, 8, &p->graph8)) return st;
        int left = n_iters;
        for (; left >= 8; left -= 8) TR_CUDA(cudaGraphLaunch(p->graph8, p->s));
        for (; left > 0; --left) TR_CUDA(cudaGraphLaunch(p->graph, p->s));
    }
    TR_CUDA(tjoin_out(p));
    return FM_OK;
}

FM_API fm_status fm_translation_merge(fm_translation *p) {
    if (fm_status st = tcheck(p)) return st;
    TR_CUDA(tjoin_in(p));
    // camera losses at the current centres of every run, then per-run normalisation
    enqueue_eval(p, 0, false, false);
    k_tr_stats<<<p->d.n_runs, TR_THREADS, 0, p->s>>>(p->d);
    k_tr_merge<<<(p->d.n_cams + TR_THREADS - 1) / TR_THREADS, TR_THREADS, 0, p->s>>>(p->d);
    TR_CUDA(cudaGetLastError());
    if (fm_status st = tcheck_errors(p)) return st;
    // one run continues from the merged centres with fresh Adam state
    p->d.n_runs = 1;
    drop_graphs(p);
    TR_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * 3 * p->d.n_cams, p->s));
    TR_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * 3 * p->d.n_cams, p->s));
    TR_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    TR_CUDA(tjoin_out(p));
    return FM_OK;
}

FM_API fm_status fm_translation_get_centres(fm_translation *p, double *o) {
    if (fm_status st = tcheck(p)) return st;
    if (!o) return tfail(FM_EINVAL, "o must not be NULL");
    TR_CUDA(tjoin_in(p));
    TR_CUDA(cudaMemcpyAsync(o, p->d.o, sizeof(double) * 3 * p->d.n_runs * p->d.n_cams, cudaMemcpyDeviceToHost,
                            p->s));
    return tcheck_errors(p);
}

FM_API fm_status fm_translation_set_centres(fm_translation *p, const double *o) {
    if (fm_status st = tcheck(p)) return st;
    if (!o) return tfail(FM_EINVAL, "o must not be NULL");
    const size_t nc3 = 3 * (size_t)p->d.n_runs * p->d.n_cams;
    if (!finite_all(o, nc3)) return tfail(FM_EINVAL, "centres must be finite");
    TR_CUDA(tjoin_in(p));
    TR_CUDA(cudaMemcpyAsync(p->d.o, o, sizeof(double) * nc3, cudaMemcpyHostToDevice, p->s));
    TR_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * nc3, p->s));
    TR_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * nc3, p->s));
    TR_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    TR_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

}  // extern "C"
