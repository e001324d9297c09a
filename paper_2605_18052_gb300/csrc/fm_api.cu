// C ABI of libfastmap: problem lifecycle, stream ordering, CUDA-graph replay of the
// optimiser iteration, error reporting. Every per-point-pair pass is a kernel in
// fm_kernels.cu / fm_layout.cu; this file only allocates, validates host arguments and
// launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fm_internal.cuh"

using namespace fm;

namespace {

thread_local std::string g_last_error;

fm_status fail(fm_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

#define FM_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? FM_ENOMEM : FM_ECUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

}  // namespace

// lets other translation units of the library report through fm_last_error
void fm_internal_set_error(const char *msg) { g_last_error = msg; }
void fm_internal_mlp_params(const fm_mlp *net, const float **master, const __nv_bfloat16 **wbf);

struct fm_problem {
    DevProblem d{};
    fm_options opt{};
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // CUDA graphs of chained iterations, by length n (key n) and of chains whose first pass is
    // fused with the reweighting (key -n)
    std::map<int, cudaGraphExec_t> chains;
    bool timing = false;
    int hist_valid = 0;                   // d.le_hist holds a previous reweighting's residuals
    double lr_focal = 1e-3;               // Adam step size of rho = log(f0/f)
    bool quad_alloc = false;              // d.qslots, d.quad, d.pair_rec allocated
    bool quad_valid = false;              // d.quad holds the form of the current weights
    cudaGraphExec_t qgraph = nullptr, qgraph8 = nullptr;  // quadratic-path iterations
    // timing events per timed pass (fm_pass_time), pairs (start, end)
    std::vector<cudaEvent_t> tev[FM_NUM_PASSES];
    size_t tev_used[FM_NUM_PASSES] = {};
    int input_was_sorted = 0;
    int64_t device_bytes = 0;
    std::vector<void *> allocs;
    double last_loss_host = 0.0;
};

namespace {

template <class T>
cudaError_t dalloc(fm_problem *p, T **ptr, size_t count) {
    const size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
    if (e == cudaSuccess) {
        p->allocs.push_back(*ptr);
        p->device_bytes += (int64_t)bytes;
    }
    return e;
}

// order the problem's stream after the caller's stream
cudaError_t join_in(fm_problem *p) {
    cudaError_t e = cudaEventRecord(p->ev_in, p->user);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->s, p->ev_in, 0);
}

// order later work of the caller's stream after the problem's stream
cudaError_t join_out(fm_problem *p) {
    cudaError_t e = cudaEventRecord(p->ev_out, p->s);
    if (e != cudaSuccess) return e;
    return cudaStreamWaitEvent(p->user, p->ev_out, 0);
}

fm_status check_device_errors(fm_problem *p) {
    unsigned err = 0;
    FM_CUDA(cudaMemcpyAsync(&err, p->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    if (err & (ERR_DEGENERATE | ERR_NONFINITE)) {
        FM_CUDA(cudaMemsetAsync(p->d.err, 0, sizeof(unsigned), p->s));
        FM_CUDA(cudaStreamSynchronize(p->s));
        return fail(FM_EDEGENERATE, (err & ERR_DEGENERATE)
                                        ? "a relative translation has zero length or the poses are not finite"
                                        : "non-finite loss or gradient");
    }
    return FM_OK;
}

bool finite_all(const double *a, size_t n) {
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(a[k])) return false;
    return true;
}

// host poses (R, t) -> device (R, c = -R^T t) and camera records
fm_status upload_poses(fm_problem *p, const double *R, const double *t) {
    const int n = p->d.n_cams;
    if (!R || !t) return fail(FM_EINVAL, "R and t must not be NULL");
    if (!finite_all(R, 9 * (size_t)n) || !finite_all(t, 3 * (size_t)n))
        return fail(FM_EINVAL, "poses must be finite");
    std::vector<double> c(3 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        const double *Rk = R + 9 * (size_t)k;
        double dev = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double dp = Rk[a] * Rk[b] + Rk[3 + a] * Rk[3 + b] + Rk[6 + a] * Rk[6 + b];
                dev = std::fmax(dev, std::fabs(dp - (a == b ? 1.0 : 0.0)));
            }
        if (dev > 1e-6) return fail(FM_EINVAL, "rotation " + std::to_string(k) + " is not orthonormal");
        for (int q = 0; q < 3; ++q)
            c[3 * k + q] = -(Rk[q] * t[3 * k] + Rk[3 + q] * t[3 * k + 1] + Rk[6 + q] * t[3 * k + 2]);
    }
    FM_CUDA(cudaMemcpyAsync(p->d.R, R, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(p->d.c, c.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, p->s));
    launch_cam_prep(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

fm_status upload_hyper(fm_problem *p) {
    const double h[6] = {p->opt.lr_rot, p->opt.lr_c, p->opt.beta1, p->opt.beta2, p->opt.adam_eps, p->lr_focal};
    FM_CUDA(cudaMemcpyAsync(p->d.hyper, h, sizeof h, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

fm_status check_options(const fm_options *o) {
    if (o->storage != FM_STORE_FP32 && o->storage != FM_STORE_FP16)
        return fail(FM_EINVAL, "storage must be FM_STORE_FP32 or FM_STORE_FP16");
    if (o->loss != FM_LOSS_IRLS && o->loss != FM_LOSS_L1)
        return fail(FM_EINVAL, "loss must be FM_LOSS_IRLS or FM_LOSS_L1");
    if (!(o->delta > 0.0) || !(o->delta < 1.0)) return fail(FM_EINVAL, "delta must be in (0, 1)");
    if (!(o->lr_rot >= 0.0) || !(o->lr_c >= 0.0) || !std::isfinite(o->lr_rot) || !std::isfinite(o->lr_c))
        return fail(FM_EINVAL, "learning rates must be finite and >= 0");
    if (!(o->beta1 >= 0.0 && o->beta1 < 1.0) || !(o->beta2 >= 0.0 && o->beta2 < 1.0))
        return fail(FM_EINVAL, "beta1 and beta2 must be in [0, 1)");
    if (!(o->adam_eps >= 0.0) || !std::isfinite(o->adam_eps)) return fail(FM_EINVAL, "adam_eps must be >= 0");
    if (o->refine_focal != 0 && o->refine_focal != 1) return fail(FM_EINVAL, "refine_focal must be 0 or 1");
    if (o->z_total < 0) return fail(FM_EINVAL, "z_total must be >= 0");
    return FM_OK;
}

// CUDA events around a pass when kernel timing is on: time_begin returns whether the pass is
// timed (then the caller launches it without programmatic serialisation and calls time_end)
bool time_begin(fm_problem *p, int pass, cudaStream_t s) {
    if (!p->timing) return false;
    std::vector<cudaEvent_t> &ev = p->tev[pass];
    if (p->tev_used[pass] + 2 > ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) break;   // the pass then runs untimed
            ev.push_back(e);
        }
    }
    if (p->tev_used[pass] + 2 > ev.size()) return false;
    cudaEventRecord(ev[p->tev_used[pass]], s);
    return true;
}

void time_end(fm_problem *p, int pass, cudaStream_t s) {
    cudaEventRecord(p->tev[pass][p->tev_used[pass] + 1], s);
    p->tev_used[pass] += 2;
}

// one optimiser iteration, chained with programmatic dependent launch: the pass over the point
// pairs, then the camera step, which also writes the geometry records of the new poses; the
// first iteration of a chain computes the geometry with a pair-setup launch, later ones find
// it written and their pass finishes the previous step's loss total and step count.
// `reweight`: the round's reweighting fused into this iteration's pass (always a first one).
void enqueue_iteration(fm_problem *p, cudaStream_t s, bool timed, bool first, bool reweight = false) {
    if (first) launch_pair_setup(p->d, s, true, false);
    const int pass = reweight ? FM_PASS_STREAM_REWEIGHT : FM_PASS_STREAM_LOSS;
    const bool t = timed && time_begin(p, pass, s);
    if (reweight) launch_stream_reweight(p->d, s, !t);
    else launch_stream_loss(p->d, s, !t, !first);
    if (t) time_end(p, pass, s);
    launch_camera_step(p->d, true, s, !t, true);
}

// `iters` chained iterations and the closing finalize launch (reweight: the first pass fused
// with the round's reweighting); `quad`: fused steps on the pre-aggregated quadratic form (one
// launch per iteration), alternating between the two camera-record buffers; after an odd count
// the finalize launch copies the records back
void enqueue_iterations(fm_problem *p, cudaStream_t s, bool timed, int iters, bool quad = false,
                        bool reweight = false) {
    if (quad) {
        for (int it = 0; it < iters; ++it) {
            const bool even = (it & 1) == 0;
            launch_quad_step(p->d, it, even ? p->d.cam : p->d.cam_alt, even ? p->d.cam_alt : p->d.cam, true, s,
                             true);
        }
        launch_finalize_n(p->d, iters, (iters & 1) ? p->d.cam_alt : nullptr, s, true);
        return;
    }
    for (int it = 0; it < iters; ++it) enqueue_iteration(p, s, timed, it == 0, reweight && it == 0);
    launch_finalize(p->d, true, s, !timed);
}

// a graph of `iters` chained iterations (reweight: the first pass fused with the reweighting)
fm_status build_graph(fm_problem *p, int iters, cudaGraphExec_t *out, bool quad = false, bool reweight = false) {
    cudaGraph_t g = nullptr;
    FM_CUDA(cudaStreamBeginCapture(p->s, cudaStreamCaptureModeThreadLocal));
    enqueue_iterations(p, p->s, false, iters, quad, reweight);
    cudaError_t e = cudaStreamEndCapture(p->s, &g);
    if (e != cudaSuccess) return fail(FM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(FM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return FM_OK;
}

// n chained iterations as CUDA graphs of whole chains (one pair-setup and one finalize launch
// per chain), built on first use and kept by length; a chain runs at most CHAIN_MAX
// iterations, and once CHAIN_CACHE lengths are kept, new lengths run as chains of 8 and 1.
// reweight: the first pass is fused with the round's reweighting.
fm_status launch_chains(fm_problem *p, int n, bool reweight) {
    constexpr int CHAIN_MAX = 64;
    constexpr size_t CHAIN_CACHE = 24;
    for (int left = n; left > 0;) {
        int len = std::min(left, CHAIN_MAX);
        if (!p->chains.count(reweight ? -len : len) && p->chains.size() >= CHAIN_CACHE) len = len >= 8 ? 8 : 1;
        const int key = reweight ? -len : len;
        auto it = p->chains.find(key);
        if (it == p->chains.end()) {
            cudaGraphExec_t g = nullptr;
            if (fm_status st = build_graph(p, len, &g, false, reweight)) return st;
            it = p->chains.emplace(key, g).first;
        }
        FM_CUDA(cudaGraphLaunch(it->second, p->s));
        left -= len;
        reweight = false;
    }
    return FM_OK;
}

void free_problem(fm_problem *p) {
    if (!p) return;
    if (p->s) cudaStreamSynchronize(p->s);
    for (void *a : p->allocs) cudaFree(a);
    for (auto &kv : p->chains) cudaGraphExecDestroy(kv.second);
    if (p->qgraph) cudaGraphExecDestroy(p->qgraph);
    if (p->qgraph8) cudaGraphExecDestroy(p->qgraph8);
    for (auto &ev : p->tev)
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->s) cudaStreamDestroy(p->s);
    delete p;
}

fm_status create_impl(fm_problem *p, int32_t n_cams, const double *R, const double *t,
                      int32_t n_pairs, const int32_t *cam_i, const int32_t *cam_j, int64_t n_pp,
                      const int32_t *pair_id, const float *x1, const float *x2,
                      int32_t pp_on_device) {
    DevProblem &d = p->d;
    d.n_cams = n_cams;
    d.n_pairs = n_pairs;
    d.n_pp = n_pp;
    d.n_pad = ((n_pp + WR - 1) / WR) * WR;
    d.n_ranges = (int)(d.n_pad / WR);
    d.storage = p->opt.storage;
    d.loss = p->opt.loss;
    d.delta = p->opt.delta;
    d.z = p->opt.z_total > 0 ? (double)p->opt.z_total : (double)n_pp;
    d.w_scale = 1.0f;
    if (d.storage == FM_STORE_FP16) d.w_scale = (float)std::exp2(std::floor(std::log2(32768.0 * p->opt.delta)));

    FM_CUDA(cudaStreamCreateWithFlags(&p->s, cudaStreamNonBlocking));
    FM_CUDA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
    FM_CUDA(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    FM_CUDA(join_in(p));

    // camera -> (pair, role) lists in pair order (host bookkeeping of the small pair table)
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

    FM_CUDA(dalloc(p, &d.R, 9 * (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.c, 3 * (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.m, 6 * (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.v, 6 * (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.rho, (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.grad_rho, (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.rho_m, (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.rho_v, (size_t)n_cams));
    d.refine_focal = p->opt.refine_focal;
    FM_CUDA(dalloc(p, &d.cam_loss, (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.hyper, 8));
    FM_CUDA(dalloc(p, &d.step, 1));
    FM_CUDA(dalloc(p, &d.cam, (size_t)CAMREC * n_cams));
    FM_CUDA(dalloc(p, &d.pair_cnt, (size_t)n_pairs));
    FM_CUDA(dalloc(p, &d.cen, (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.cam_i, (size_t)n_pairs));
    FM_CUDA(dalloc(p, &d.cam_j, (size_t)n_pairs));
    FM_CUDA(dalloc(p, &d.pair_off, (size_t)n_pairs + 1));
    FM_CUDA(dalloc(p, &d.range_pair, (size_t)d.n_ranges));
    FM_CUDA(dalloc(p, &d.cam_off, (size_t)n_cams + 1));
    FM_CUDA(dalloc(p, &d.cam_ent, 2 * (size_t)n_pairs));
    if (d.storage == FM_STORE_FP32) {
        float4 *kp;
        float *w;
        FM_CUDA(dalloc(p, &kp, (size_t)d.n_pad));
        FM_CUDA(dalloc(p, &w, (size_t)d.n_pad));
        d.kp = kp;
        d.w = w;
    } else {
        uint2 *kp;
        __half *w;
        FM_CUDA(dalloc(p, &kp, (size_t)d.n_pad));
        FM_CUDA(dalloc(p, &w, (size_t)d.n_pad));
        d.kp = kp;
        d.w = w;
    }
    FM_CUDA(dalloc(p, &d.score, (size_t)d.n_pad));
    FM_CUDA(dalloc(p, &d.le_hist, (size_t)d.n_pad));
    {
        float4 *ps;
        FM_CUDA(dalloc(p, &ps, (size_t)n_pairs));
        d.pstat = reinterpret_cast<float *>(ps);
    }
    FM_CUDA(dalloc(p, &d.geo, (size_t)GEO * n_pairs));
    FM_CUDA(dalloc(p, &d.slots, (size_t)SLOT * ((size_t)n_pairs + d.n_ranges)));
    FM_CUDA(dalloc(p, &d.pair_grad, (size_t)PG * n_pairs));
    FM_CUDA(dalloc(p, &d.grad, 6 * (size_t)n_cams));
    FM_CUDA(dalloc(p, &d.loss_out, 1));
    FM_CUDA(dalloc(p, &d.err, 1));
    FM_CUDA(dalloc(p, &d.counter, 1));
    d.perm = nullptr;
    d.fbuf = nullptr;

    FM_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), p->s));
    FM_CUDA(cudaMemsetAsync(d.m, 0, sizeof(float) * 6 * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.v, 0, sizeof(float) * 6 * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.rho, 0, sizeof(double) * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.grad_rho, 0, sizeof(double) * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.rho_m, 0, sizeof(float) * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.rho_v, 0, sizeof(float) * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.step, 0, sizeof(long long), p->s));
    FM_CUDA(cudaMemsetAsync(d.cen, 0, sizeof(float2) * n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(d.geo, 0, sizeof(float) * GEO * n_pairs, p->s));
    FM_CUDA(cudaMemsetAsync(d.pair_cnt, 0, sizeof(unsigned) * n_pairs, p->s));
    FM_CUDA(cudaMemcpyAsync(d.cam_i, cam_i, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(d.cam_j, cam_j, sizeof(int) * n_pairs, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(d.cam_off, cam_off.data(), sizeof(int) * (n_cams + 1), cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(d.cam_ent, cam_ent.data(), sizeof(int) * 2 * n_pairs, cudaMemcpyHostToDevice, p->s));

    // point pairs on the device (temporaries when they come from the host)
    const int *d_pid = pair_id;
    const float2 *d_x1 = reinterpret_cast<const float2 *>(x1);
    const float2 *d_x2 = reinterpret_cast<const float2 *>(x2);
    int *t_pid = nullptr;
    float2 *t_x1 = nullptr, *t_x2 = nullptr;
    if (!pp_on_device) {
        FM_CUDA(cudaMallocAsync(&t_pid, sizeof(int) * n_pp, p->s));
        FM_CUDA(cudaMallocAsync(&t_x1, sizeof(float2) * n_pp, p->s));
        FM_CUDA(cudaMallocAsync(&t_x2, sizeof(float2) * n_pp, p->s));
        FM_CUDA(cudaMemcpyAsync(t_pid, pair_id, sizeof(int) * n_pp, cudaMemcpyHostToDevice, p->s));
        FM_CUDA(cudaMemcpyAsync(t_x1, x1, sizeof(float2) * n_pp, cudaMemcpyHostToDevice, p->s));
        FM_CUDA(cudaMemcpyAsync(t_x2, x2, sizeof(float2) * n_pp, cudaMemcpyHostToDevice, p->s));
        d_pid = t_pid;
        d_x1 = t_x1;
        d_x2 = t_x2;
    }
    auto release_temps = [&]() {
        if (t_pid) cudaFreeAsync(t_pid, p->s);
        if (t_x1) cudaFreeAsync(t_x1, p->s);
        if (t_x2) cudaFreeAsync(t_x2, p->s);
        t_pid = nullptr;
        t_x1 = t_x2 = nullptr;
    };

    launch_validate(d_pid, d_x1, d_x2, n_pp, n_pairs, d.err, p->s);
    FM_CUDA(cudaGetLastError());
    unsigned err = 0;
    FM_CUDA(cudaMemcpyAsync(&err, d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    if (err & (ERR_PAIR_RANGE | ERR_COORD)) {
        release_temps();
        cudaStreamSynchronize(p->s);
        return fail(FM_EINVAL, (err & ERR_PAIR_RANGE) ? "pair_id out of range [0, n_pairs)"
                                                       : "keypoint coordinates must be finite with |x| <= 8");
    }
    p->input_was_sorted = (err & ERR_UNSORTED) ? 0 : 1;

    const int *keys = d_pid;
    int *sorted_keys = nullptr;
    if (!p->input_was_sorted) {
        FM_CUDA(dalloc(p, &d.perm, (size_t)n_pp));
        FM_CUDA(cudaMallocAsync(&sorted_keys, sizeof(int) * n_pp, p->s));
        FM_CUDA(sort_by_pair(d_pid, n_pp, n_pairs, sorted_keys, d.perm, p->s));
        keys = sorted_keys;
    }
    launch_pair_offsets(keys, n_pp, n_pairs, d.pair_off, d.err, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(&err, d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    if (err & ERR_EMPTY_PAIR) {
        if (sorted_keys) cudaFreeAsync(sorted_keys, p->s);
        release_temps();
        cudaStreamSynchronize(p->s);
        return fail(FM_EINVAL, "every image pair needs at least one point pair");
    }
    launch_range_pairs(d.pair_off, n_pairs, d.n_ranges, d.range_pair, p->s);
    if (d.storage == FM_STORE_FP16) {
        unsigned long long *sums = nullptr;
        FM_CUDA(cudaMallocAsync(&sums, sizeof(unsigned long long) * 2 * n_cams, p->s));
        launch_centroids(d, keys, d_x1, d_x2, sums, p->s);
        FM_CUDA(cudaFreeAsync(sums, p->s));
    }
    launch_pack(d, keys, d_x1, d_x2, p->s);
    launch_fill_weights(d, 1.0f, p->s);
    launch_fill_half(d.score, d.n_pad, 0.5f, p->s);
    launch_fill_half(d.le_hist, d.n_pad, 0.0f, p->s);
    FM_CUDA(cudaGetLastError());
    if (sorted_keys) FM_CUDA(cudaFreeAsync(sorted_keys, p->s));
    release_temps();
    FM_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));

    fm_status st = upload_poses(p, R, t);
    if (st != FM_OK) return st;
    st = upload_hyper(p);
    if (st != FM_OK) return st;
    FM_CUDA(join_out(p));
    return FM_OK;
}

fm_status check_problem(const fm_problem *p) {
    if (!p) return fail(FM_EINVAL, "problem is NULL");
    return FM_OK;
}

}  // namespace

// =================================== C ABI ===================================================
extern "C" {

FM_API void fm_default_options(fm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->storage = FM_STORE_FP32;
    o->loss = FM_LOSS_IRLS;
    o->delta = 1e-6;
    o->lr_rot = 1e-2;
    o->lr_c = 1e-2;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->adam_eps = 1e-12;
    o->use_graph = 1;
    o->refine_focal = 0;
    o->z_total = 0;
}

FM_API fm_status fm_create_problem(int32_t n_cams, const double *R, const double *t,
                                   int32_t n_pairs, const int32_t *cam_i, const int32_t *cam_j,
                                   int64_t n_pp, const int32_t *pair_id, const float *x1,
                                   const float *x2, int32_t pp_on_device, const fm_options *opt,
                                   void *stream, fm_problem **out) {
    if (!out) return fail(FM_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n_cams < 2) return fail(FM_EINVAL, "n_cams must be >= 2");
    if (n_pairs < 1) return fail(FM_EINVAL, "n_pairs must be >= 1");
    if (n_pp < 1 || n_pp >= (int64_t)(2147483647ll - 65536)) return fail(FM_EINVAL, "n_pp out of range");
    if (n_pairs > n_pp) return fail(FM_EINVAL, "every image pair needs at least one point pair");
    if (!R || !t || !cam_i || !cam_j || !pair_id || !x1 || !x2)
        return fail(FM_EINVAL, "input pointers must not be NULL");
    if (pp_on_device != 0 && pp_on_device != 1) return fail(FM_EINVAL, "pp_on_device must be 0 or 1");
    for (int n = 0; n < n_pairs; ++n) {
        if (cam_i[n] < 0 || cam_i[n] >= n_cams || cam_j[n] < 0 || cam_j[n] >= n_cams)
            return fail(FM_EINVAL, "camera index of pair " + std::to_string(n) + " out of range");
        if (cam_i[n] == cam_j[n]) return fail(FM_EINVAL, "pair " + std::to_string(n) + " has cam_i == cam_j");
    }
    fm_options o;
    if (opt) o = *opt;
    else fm_default_options(&o);
    fm_status st = check_options(&o);
    if (st != FM_OK) return st;
    fm_problem *p = new (std::nothrow) fm_problem();
    if (!p) return fail(FM_ENOMEM, "host allocation failed");
    p->opt = o;
    p->user = static_cast<cudaStream_t>(stream);
    st = create_impl(p, n_cams, R, t, n_pairs, cam_i, cam_j, n_pp, pair_id, x1, x2, pp_on_device);
    if (st != FM_OK) {
        const std::string msg = g_last_error;
        free_problem(p);
        g_last_error = msg;
        return st;
    }
    *out = p;
    return FM_OK;
}

FM_API void fm_destroy_problem(fm_problem *p) { free_problem(p); }

FM_API fm_status fm_problem_info(const fm_problem *p, fm_info *info) {
    if (fm_status st = check_problem(p)) return st;
    if (!info) return fail(FM_EINVAL, "info must not be NULL");
    std::memset(info, 0, sizeof *info);
    info->n_cams = p->d.n_cams;
    info->n_pairs = p->d.n_pairs;
    info->n_pp = p->d.n_pp;
    info->storage = p->d.storage;
    info->loss = p->d.loss;
    info->n_warp_ranges = p->d.n_ranges;
    const int64_t per_pp = p->d.storage == FM_STORE_FP32 ? 16 : 8;
    const int64_t per_w = p->d.loss == FM_LOSS_IRLS ? (p->d.storage == FM_STORE_FP32 ? 4 : 2) : 0;
    info->stream_bytes = p->d.n_pp * (per_pp + per_w);
    info->device_bytes = p->device_bytes;
    info->input_was_sorted = p->input_was_sorted;
    return FM_OK;
}

FM_API fm_status fm_get_poses(fm_problem *p, double *R, double *t) {
    if (fm_status st = check_problem(p)) return st;
    if (!R || !t) return fail(FM_EINVAL, "R and t must not be NULL");
    const int n = p->d.n_cams;
    std::vector<double> c(3 * (size_t)n);
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(R, p->d.R, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaMemcpyAsync(c.data(), p->d.c, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, p->s));
    if (fm_status st = check_device_errors(p)) return st;
    for (int k = 0; k < n; ++k) {
        const double *Rk = R + 9 * (size_t)k;
        for (int a = 0; a < 3; ++a)
            t[3 * k + a] = -(Rk[3 * a] * c[3 * k] + Rk[3 * a + 1] * c[3 * k + 1] + Rk[3 * a + 2] * c[3 * k + 2]);
    }
    return FM_OK;
}

FM_API fm_status fm_set_poses(fm_problem *p, const double *R, const double *t) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(join_in(p));
    fm_status st = upload_poses(p, R, t);
    if (st != FM_OK) return st;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_get_params(fm_problem *p, double *R, double *c) {
    if (fm_status st = check_problem(p)) return st;
    if (!R || !c) return fail(FM_EINVAL, "R and c must not be NULL");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(R, p->d.R, sizeof(double) * 9 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaMemcpyAsync(c, p->d.c, sizeof(double) * 3 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return check_device_errors(p);
}

FM_API fm_status fm_set_params(fm_problem *p, const double *R, const double *c) {
    if (fm_status st = check_problem(p)) return st;
    if (!R || !c) return fail(FM_EINVAL, "R and c must not be NULL");
    const int n = p->d.n_cams;
    if (!finite_all(R, 9 * (size_t)n) || !finite_all(c, 3 * (size_t)n))
        return fail(FM_EINVAL, "parameters must be finite");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(p->d.R, R, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(p->d.c, c, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, p->s));
    launch_cam_prep(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaStreamSynchronize(p->s));
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_set_params_device(fm_problem *p, const double *d_R, const double *d_c) {
    if (fm_status st = check_problem(p)) return st;
    if (!d_R || !d_c) return fail(FM_EINVAL, "d_R and d_c must not be NULL");
    const int n = p->d.n_cams;
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(p->d.R, d_R, sizeof(double) * 9 * n, cudaMemcpyDeviceToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(p->d.c, d_c, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, p->s));
    launch_cam_prep(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_set_weights(fm_problem *p, const float *w, int32_t on_device) {
    if (fm_status st = check_problem(p)) return st;
    if (!w) return fail(FM_EINVAL, "w must not be NULL");
    if (on_device != 0 && on_device != 1) return fail(FM_EINVAL, "on_device must be 0 or 1");
    FM_CUDA(join_in(p));
    const float *src = w;
    float *tmp = nullptr;
    if (!on_device) {
        FM_CUDA(cudaMallocAsync(&tmp, sizeof(float) * p->d.n_pp, p->s));
        FM_CUDA(cudaMemcpyAsync(tmp, w, sizeof(float) * p->d.n_pp, cudaMemcpyHostToDevice, p->s));
        src = tmp;
    }
    launch_set_weights(p->d, src, p->s);
    p->quad_valid = false;
    FM_CUDA(cudaGetLastError());
    if (tmp) FM_CUDA(cudaFreeAsync(tmp, p->s));
    unsigned err = 0;
    FM_CUDA(cudaMemcpyAsync(&err, p->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    if (err & ERR_WEIGHT) {
        unsigned keep = err & ~ERR_WEIGHT;
        FM_CUDA(cudaMemcpyAsync(p->d.err, &keep, sizeof(unsigned), cudaMemcpyHostToDevice, p->s));
        FM_CUDA(cudaStreamSynchronize(p->s));
        return fail(FM_EINVAL, "weights must be finite and in [0, 1/delta]; offending weights were set to 0");
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_get_weights(fm_problem *p, float *w) {
    if (fm_status st = check_problem(p)) return st;
    if (!w) return fail(FM_EINVAL, "w must not be NULL");
    FM_CUDA(join_in(p));
    float *tmp = nullptr;
    FM_CUDA(cudaMallocAsync(&tmp, sizeof(float) * p->d.n_pp, p->s));
    launch_get_weights(p->d, tmp, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(w, tmp, sizeof(float) * p->d.n_pp, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaFreeAsync(tmp, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

FM_API fm_status fm_set_scores(fm_problem *p, const float *score, int32_t on_device) {
    if (fm_status st = check_problem(p)) return st;
    if (!score) return fail(FM_EINVAL, "score must not be NULL");
    if (on_device != 0 && on_device != 1) return fail(FM_EINVAL, "on_device must be 0 or 1");
    FM_CUDA(join_in(p));
    const float *src = score;
    float *tmp = nullptr;
    if (!on_device) {
        FM_CUDA(cudaMallocAsync(&tmp, sizeof(float) * p->d.n_pp, p->s));
        FM_CUDA(cudaMemcpyAsync(tmp, score, sizeof(float) * p->d.n_pp, cudaMemcpyHostToDevice, p->s));
        src = tmp;
    }
    launch_set_scores(p->d, src, p->s);
    FM_CUDA(cudaGetLastError());
    if (tmp) FM_CUDA(cudaFreeAsync(tmp, p->s));
    unsigned err = 0;
    FM_CUDA(cudaMemcpyAsync(&err, p->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    if (err & ERR_WEIGHT) {
        unsigned keep = err & ~ERR_WEIGHT;
        FM_CUDA(cudaMemcpyAsync(p->d.err, &keep, sizeof(unsigned), cudaMemcpyHostToDevice, p->s));
        FM_CUDA(cudaStreamSynchronize(p->s));
        return fail(FM_EINVAL, "scores must be in [0, 1]; offending scores were set to 0.5");
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_reset_history(fm_problem *p) {
    if (fm_status st = check_problem(p)) return st;
    p->hist_valid = 0;
    return FM_OK;
}

FM_API fm_status fm_collect_features(fm_problem *p, double tau, int32_t round, void *d_features) {
    if (fm_status st = check_problem(p)) return st;
    if (!d_features) return fail(FM_EINVAL, "d_features must not be NULL");
    if (!(tau > 0.0) || std::isinf(tau)) return fail(FM_EINVAL, "tau must be finite and > 0");
    if (round < 0) return fail(FM_EINVAL, "round must be >= 0");
    FM_CUDA(join_in(p));
    launch_pair_setup(p->d, p->s);
    launch_pair_stats(p->d, (float)tau, p->s);
    launch_collect_features(p->d, (float)tau, round, p->hist_valid, static_cast<__nv_bfloat16 *>(d_features), p->s);
    FM_CUDA(cudaGetLastError());
    p->hist_valid = 1;
    if (fm_status st = check_device_errors(p)) return st;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_learned_weights(fm_problem *p, const fm_mlp *net, double tau, double tau_cap,
                                    int32_t round, int64_t *n_active) {
    if (fm_status st = check_problem(p)) return st;
    if (!net) return fail(FM_EINVAL, "net must not be NULL");
    if (!(tau > 0.0) || std::isinf(tau)) return fail(FM_EINVAL, "tau must be finite and > 0");
    if (std::isnan(tau_cap) || tau_cap < 0.0) return fail(FM_EINVAL, "tau_cap must be >= 0 (may be +inf)");
    if (round < 0) return fail(FM_EINVAL, "round must be >= 0");
    const float *master = nullptr;
    const __nv_bfloat16 *wbf = nullptr;
    fm_internal_mlp_params(net, &master, &wbf);
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(unsigned long long), p->s));
    launch_pair_setup(p->d, p->s);
    launch_pair_stats(p->d, (float)tau, p->s);
    launch_learned_weights(p->d, master, wbf, (float)tau, std::isinf(tau_cap) ? INFINITY : (float)tau_cap, round,
                           p->hist_valid, p->s);
    p->quad_valid = false;
    FM_CUDA(cudaGetLastError());
    p->hist_valid = 1;
    unsigned long long cnt = 0;
    FM_CUDA(cudaMemcpyAsync(&cnt, p->d.counter, sizeof cnt, cudaMemcpyDeviceToHost, p->s));
    if (fm_status st = check_device_errors(p)) return st;
    if (n_active) *n_active = (int64_t)cnt;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_step_learned(fm_problem *p, const fm_mlp *net, double tau, double tau_cap, int32_t round,
                                 int32_t n_iters, int64_t *n_active) {
    if (fm_status st = check_problem(p)) return st;
    if (!net) return fail(FM_EINVAL, "net must not be NULL");
    if (!(tau > 0.0) || std::isinf(tau)) return fail(FM_EINVAL, "tau must be finite and > 0");
    if (std::isnan(tau_cap) || tau_cap < 0.0) return fail(FM_EINVAL, "tau_cap must be >= 0 (may be +inf)");
    if (round < 0) return fail(FM_EINVAL, "round must be >= 0");
    if (n_iters < 1) return fail(FM_EINVAL, "n_iters must be >= 1");
    if (p->d.loss != FM_LOSS_IRLS) return fail(FM_EINVAL, "the fused reweighting needs the IRLS objective");
    const float *master = nullptr;
    const __nv_bfloat16 *wbf = nullptr;
    fm_internal_mlp_params(net, &master, &wbf);
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(unsigned long long), p->s));
    launch_pair_setup(p->d, p->s);
    const bool ts = time_begin(p, FM_PASS_PAIR_STATS, p->s);
    launch_pair_stats(p->d, (float)tau, p->s);
    if (ts) time_end(p, FM_PASS_PAIR_STATS, p->s);
    const bool tl = time_begin(p, FM_PASS_LEARNED_LOSS, p->s);
    launch_learned_loss(p->d, master, wbf, (float)tau, std::isinf(tau_cap) ? INFINITY : (float)tau_cap, round,
                        p->hist_valid, p->s, false);
    if (tl) time_end(p, FM_PASS_LEARNED_LOSS, p->s);
    launch_camera_step(p->d, true, p->s, !tl);
    launch_finalize(p->d, true, p->s, !tl);
    FM_CUDA(cudaGetLastError());
    p->quad_valid = false;
    p->hist_valid = 1;
    unsigned long long cnt = 0;
    if (n_active) FM_CUDA(cudaMemcpyAsync(&cnt, p->d.counter, sizeof cnt, cudaMemcpyDeviceToHost, p->s));
    if (n_iters > 1)
        if (fm_status st = fm_step(p, n_iters - 1)) return st;
    if (n_active) {
        if (fm_status st = check_device_errors(p)) return st;
        *n_active = (int64_t)cnt;
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_irls_weights(fm_problem *p, double tau, int64_t *n_active) {
    if (fm_status st = check_problem(p)) return st;
    if (std::isnan(tau) || tau < 0.0) return fail(FM_EINVAL, "tau must be >= 0 (may be +inf)");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(unsigned long long), p->s));
    launch_pair_setup(p->d, p->s);
    const float tf = std::isinf(tau) ? INFINITY : (float)tau;
    launch_irls_weights(p->d, tf, p->s);
    p->quad_valid = false;
    FM_CUDA(cudaGetLastError());
    unsigned long long cnt = 0;
    FM_CUDA(cudaMemcpyAsync(&cnt, p->d.counter, sizeof cnt, cudaMemcpyDeviceToHost, p->s));
    if (fm_status st = check_device_errors(p)) return st;
    if (n_active) *n_active = (int64_t)cnt;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_loss_grad_device(fm_problem *p, double *d_loss, double *d_grad) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(join_in(p));
    launch_pair_setup(p->d, p->s);
    launch_stream_loss(p->d, p->s);
    launch_camera_step(p->d, false, p->s);
    launch_finalize(p->d, false, p->s);
    FM_CUDA(cudaGetLastError());
    if (d_loss) FM_CUDA(cudaMemcpyAsync(d_loss, p->d.loss_out, sizeof(double), cudaMemcpyDeviceToDevice, p->s));
    if (d_grad)
        FM_CUDA(cudaMemcpyAsync(d_grad, p->d.grad, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyDeviceToDevice, p->s));
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_loss_grad(fm_problem *p, double *loss, double *grad) {
    if (fm_status st = check_problem(p)) return st;
    if (!loss) return fail(FM_EINVAL, "loss must not be NULL");
    FM_CUDA(join_in(p));
    launch_pair_setup(p->d, p->s);
    launch_stream_loss(p->d, p->s);
    launch_camera_step(p->d, false, p->s);
    launch_finalize(p->d, false, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(loss, p->d.loss_out, sizeof(double), cudaMemcpyDeviceToHost, p->s));
    if (grad)
        FM_CUDA(cudaMemcpyAsync(grad, p->d.grad, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return check_device_errors(p);
}

FM_API fm_status fm_residuals(fm_problem *p, float *eps) {
    if (fm_status st = check_problem(p)) return st;
    if (!eps) return fail(FM_EINVAL, "eps must not be NULL");
    FM_CUDA(join_in(p));
    float *sorted = nullptr, *ordered = nullptr;
    FM_CUDA(cudaMallocAsync(&sorted, sizeof(float) * p->d.n_pp, p->s));
    FM_CUDA(cudaMallocAsync(&ordered, sizeof(float) * p->d.n_pp, p->s));
    launch_pair_setup(p->d, p->s);
    launch_residuals(p->d, sorted, p->s);
    launch_unpermute(p->d, sorted, ordered, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(eps, ordered, sizeof(float) * p->d.n_pp, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaFreeAsync(sorted, p->s));
    FM_CUDA(cudaFreeAsync(ordered, p->s));
    return check_device_errors(p);
}

FM_API fm_status fm_step(fm_problem *p, int32_t n_iters) {
    if (fm_status st = check_problem(p)) return st;
    if (n_iters < 0) return fail(FM_EINVAL, "n_iters must be >= 0");
    if (n_iters == 0) return FM_OK;
    FM_CUDA(join_in(p));
    if (p->timing || !p->opt.use_graph) {
        enqueue_iterations(p, p->s, p->timing, n_iters);
        FM_CUDA(cudaGetLastError());
    } else if (fm_status st = launch_chains(p, n_iters, false)) {
        return st;
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_step_irls(fm_problem *p, double tau, int32_t n_iters, int64_t *n_active) {
    if (fm_status st = check_problem(p)) return st;
    if (std::isnan(tau) || tau < 0.0) return fail(FM_EINVAL, "tau must be >= 0 (may be +inf)");
    if (n_iters < 1) return fail(FM_EINVAL, "n_iters must be >= 1");
    if (p->d.loss != FM_LOSS_IRLS) return fail(FM_EINVAL, "the fused reweighting needs the IRLS objective");
    FM_CUDA(join_in(p));
    const double tv = std::isinf(tau) ? INFINITY : (double)(float)tau;
    FM_CUDA(cudaMemcpyAsync(p->d.hyper + 6, &tv, sizeof tv, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(unsigned long long), p->s));
    p->quad_valid = false;
    if (p->timing || !p->opt.use_graph) {
        enqueue_iterations(p, p->s, p->timing, n_iters, false, true);
        FM_CUDA(cudaGetLastError());
    } else if (fm_status st = launch_chains(p, n_iters, true)) {
        return st;
    }
    unsigned long long cnt = 0;
    if (n_active) FM_CUDA(cudaMemcpyAsync(&cnt, p->d.counter, sizeof cnt, cudaMemcpyDeviceToHost, p->s));
    if (n_active) {
        if (fm_status st = check_device_errors(p)) return st;
        *n_active = (int64_t)cnt;
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_last_loss(fm_problem *p, double *loss) {
    if (fm_status st = check_problem(p)) return st;
    if (!loss) return fail(FM_EINVAL, "loss must not be NULL");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(loss, p->d.loss_out, sizeof(double), cudaMemcpyDeviceToHost, p->s));
    return check_device_errors(p);
}

FM_API fm_status fm_apply_gradient(fm_problem *p, const double *grad, int32_t on_device) {
    if (fm_status st = check_problem(p)) return st;
    if (!grad) return fail(FM_EINVAL, "grad must not be NULL");
    if (on_device != 0 && on_device != 1) return fail(FM_EINVAL, "on_device must be 0 or 1");
    if (!on_device && !finite_all(grad, 6 * (size_t)p->d.n_cams)) return fail(FM_EINVAL, "gradient must be finite");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(p->d.grad, grad, sizeof(double) * 6 * p->d.n_cams,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->s));
    launch_apply_gradient(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    if (!on_device) FM_CUDA(cudaStreamSynchronize(p->s));   // the host buffer may be reused at once
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_set_learning_rate(fm_problem *p, double lr_rot, double lr_c) {
    if (fm_status st = check_problem(p)) return st;
    if (!(lr_rot >= 0.0) || !(lr_c >= 0.0) || !std::isfinite(lr_rot) || !std::isfinite(lr_c))
        return fail(FM_EINVAL, "learning rates must be finite and >= 0");
    p->opt.lr_rot = lr_rot;
    p->opt.lr_c = lr_c;
    FM_CUDA(join_in(p));
    return upload_hyper(p);
}

FM_API fm_status fm_reset_optimizer(fm_problem *p) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemsetAsync(p->d.m, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.v, 0, sizeof(float) * 6 * p->d.n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.rho_m, 0, sizeof(float) * p->d.n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.rho_v, 0, sizeof(float) * p->d.n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.step, 0, sizeof(long long), p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

FM_API fm_status fm_get_state(fm_problem *p, double *m, double *v, int64_t *step) {
    if (fm_status st = check_problem(p)) return st;
    if (!m || !v || !step) return fail(FM_EINVAL, "m, v and step must not be NULL");
    long long s = 0;
    const size_t n6 = 6 * (size_t)p->d.n_cams;
    std::vector<float> mf(n6), vf(n6);
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(mf.data(), p->d.m, sizeof(float) * n6, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaMemcpyAsync(vf.data(), p->d.v, sizeof(float) * n6, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaMemcpyAsync(&s, p->d.step, sizeof s, cudaMemcpyDeviceToHost, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    for (size_t k = 0; k < n6; ++k) {
        m[k] = mf[k];
        v[k] = vf[k];
    }
    *step = s;
    return FM_OK;
}

FM_API fm_status fm_set_state(fm_problem *p, const double *m, const double *v, int64_t step) {
    if (fm_status st = check_problem(p)) return st;
    if (!m || !v) return fail(FM_EINVAL, "m and v must not be NULL");
    if (step < 0) return fail(FM_EINVAL, "step must be >= 0");
    if (!finite_all(m, 6 * (size_t)p->d.n_cams) || !finite_all(v, 6 * (size_t)p->d.n_cams))
        return fail(FM_EINVAL, "optimiser state must be finite");
    for (size_t k = 0; k < 6 * (size_t)p->d.n_cams; ++k)
        if (v[k] < 0.0) return fail(FM_EINVAL, "second moments must be >= 0");
    const long long s = step;
    const size_t n6 = 6 * (size_t)p->d.n_cams;
    std::vector<float> mf(n6), vf(n6);
    for (size_t k = 0; k < n6; ++k) {
        mf[k] = (float)m[k];
        vf[k] = (float)v[k];
    }
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(p->d.m, mf.data(), sizeof(float) * n6, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(p->d.v, vf.data(), sizeof(float) * n6, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemcpyAsync(p->d.step, &s, sizeof s, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

// ---- focal refinement ----------------------------------------------------------------------------
FM_API fm_status fm_set_focal_learning_rate(fm_problem *p, double lr) {
    if (fm_status st = check_problem(p)) return st;
    if (!(lr >= 0.0) || !std::isfinite(lr)) return fail(FM_EINVAL, "lr must be finite and >= 0");
    p->lr_focal = lr;
    FM_CUDA(join_in(p));
    return upload_hyper(p);
}

FM_API fm_status fm_get_focal_scales(fm_problem *p, double *s) {
    if (fm_status st = check_problem(p)) return st;
    if (!s) return fail(FM_EINVAL, "s must not be NULL");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(s, p->d.rho, sizeof(double) * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    if (fm_status st = check_device_errors(p)) return st;
    for (int k = 0; k < p->d.n_cams; ++k) s[k] = std::exp(s[k]);
    return FM_OK;
}

FM_API fm_status fm_set_focal_scales(fm_problem *p, const double *s) {
    if (fm_status st = check_problem(p)) return st;
    if (!s) return fail(FM_EINVAL, "s must not be NULL");
    std::vector<double> rho(p->d.n_cams);
    for (int k = 0; k < p->d.n_cams; ++k) {
        if (!(s[k] > 0.0) || !std::isfinite(s[k])) return fail(FM_EINVAL, "scales must be finite and > 0");
        rho[k] = std::log(s[k]);
    }
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(p->d.rho, rho.data(), sizeof(double) * p->d.n_cams, cudaMemcpyHostToDevice, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.rho_m, 0, sizeof(float) * p->d.n_cams, p->s));
    FM_CUDA(cudaMemsetAsync(p->d.rho_v, 0, sizeof(float) * p->d.n_cams, p->s));
    launch_cam_prep(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    p->quad_valid = false;
    FM_CUDA(cudaStreamSynchronize(p->s));
    return FM_OK;
}

FM_API fm_status fm_get_focal_gradient(fm_problem *p, double *g) {
    if (fm_status st = check_problem(p)) return st;
    if (!g) return fail(FM_EINVAL, "g must not be NULL");
    FM_CUDA(join_in(p));
    FM_CUDA(cudaMemcpyAsync(g, p->d.grad_rho, sizeof(double) * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return check_device_errors(p);
}

// ---- pre-aggregated quadratic form ------------------------------------------------------------
namespace {

fm_status quad_prepare(fm_problem *p) {
    if (p->d.loss != FM_LOSS_IRLS) return fail(FM_EINVAL, "the quadratic form needs the IRLS objective");
    if (p->quad_alloc) return FM_OK;
    FM_CUDA(dalloc(p, &p->d.qslots, (size_t)QSLOT * ((size_t)p->d.n_pairs + p->d.n_ranges)));
    FM_CUDA(dalloc(p, &p->d.quad, (size_t)QREC * p->d.n_pairs));
    FM_CUDA(dalloc(p, &p->d.cam_alt, (size_t)CAMREC * p->d.n_cams));
    p->quad_alloc = true;
    return FM_OK;
}

fm_status quad_check(fm_problem *p) {
    if (p->d.loss != FM_LOSS_IRLS) return fail(FM_EINVAL, "the quadratic form needs the IRLS objective");
    if (!p->quad_valid)
        return fail(FM_EINVAL, "no quadratic form for the current weights (call fm_preaggregate first)");
    return FM_OK;
}

}  // namespace

FM_API fm_status fm_preaggregate(fm_problem *p) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(join_in(p));
    if (fm_status st = quad_prepare(p)) return st;
    launch_pair_setup(p->d, p->s);
    const bool tq = time_begin(p, FM_PASS_QUAD_ACCUMULATE, p->s);
    launch_quad_accumulate(p->d, -1.f, p->s);
    if (tq) time_end(p, FM_PASS_QUAD_ACCUMULATE, p->s);
    launch_quad_combine(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    p->quad_valid = true;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_irls_preaggregate(fm_problem *p, double tau, int64_t *n_active) {
    if (fm_status st = check_problem(p)) return st;
    if (std::isnan(tau) || tau < 0.0) return fail(FM_EINVAL, "tau must be >= 0 (may be +inf)");
    FM_CUDA(join_in(p));
    if (fm_status st = quad_prepare(p)) return st;
    FM_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(unsigned long long), p->s));
    launch_pair_setup(p->d, p->s);
    const bool tq = time_begin(p, FM_PASS_QUAD_ACCUMULATE, p->s);
    launch_quad_accumulate(p->d, std::isinf(tau) ? INFINITY : (float)tau, p->s);
    if (tq) time_end(p, FM_PASS_QUAD_ACCUMULATE, p->s);
    launch_quad_combine(p->d, p->s);
    FM_CUDA(cudaGetLastError());
    p->quad_valid = true;
    unsigned long long cnt = 0;
    FM_CUDA(cudaMemcpyAsync(&cnt, p->d.counter, sizeof cnt, cudaMemcpyDeviceToHost, p->s));
    if (fm_status st = check_device_errors(p)) return st;
    if (n_active) *n_active = (int64_t)cnt;
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_loss_grad_quadratic(fm_problem *p, double *loss, double *grad) {
    if (fm_status st = check_problem(p)) return st;
    if (!loss) return fail(FM_EINVAL, "loss must not be NULL");
    if (fm_status st = quad_check(p)) return st;
    FM_CUDA(join_in(p));
    launch_quad_step(p->d, 0, p->d.cam, p->d.cam_alt, false, p->s, false);
    launch_finalize(p->d, false, p->s);
    FM_CUDA(cudaGetLastError());
    FM_CUDA(cudaMemcpyAsync(loss, p->d.loss_out, sizeof(double), cudaMemcpyDeviceToHost, p->s));
    if (grad)
        FM_CUDA(cudaMemcpyAsync(grad, p->d.grad, sizeof(double) * 6 * p->d.n_cams, cudaMemcpyDeviceToHost, p->s));
    return check_device_errors(p);
}

FM_API fm_status fm_step_quadratic(fm_problem *p, int32_t n_iters) {
    if (fm_status st = check_problem(p)) return st;
    if (n_iters < 0) return fail(FM_EINVAL, "n_iters must be >= 0");
    if (fm_status st = quad_check(p)) return st;
    if (n_iters == 0) return FM_OK;
    FM_CUDA(join_in(p));
    if (!p->opt.use_graph) {
        enqueue_iterations(p, p->s, false, n_iters, true);
        FM_CUDA(cudaGetLastError());
    } else {
        if (!p->qgraph) {
            fm_status st = build_graph(p, 1, &p->qgraph, true);
            if (st != FM_OK) return st;
        }
        if (n_iters >= 8 && !p->qgraph8) {
            fm_status st = build_graph(p, 8, &p->qgraph8, true);
            if (st != FM_OK) return st;
        }
        int left = n_iters;
        for (; left >= 8; left -= 8) FM_CUDA(cudaGraphLaunch(p->qgraph8, p->s));
        for (; left > 0; --left) FM_CUDA(cudaGraphLaunch(p->qgraph, p->s));
    }
    FM_CUDA(join_out(p));
    return FM_OK;
}

FM_API fm_status fm_synchronize(fm_problem *p) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(join_in(p));
    return check_device_errors(p);
}

FM_API fm_status fm_enable_kernel_timing(fm_problem *p, int32_t enable) {
    if (fm_status st = check_problem(p)) return st;
    FM_CUDA(cudaStreamSynchronize(p->s));
    p->timing = enable != 0;
    for (size_t &u : p->tev_used) u = 0;
    return FM_OK;
}

FM_API fm_status fm_pass_time(fm_problem *p, int32_t pass, double *ms, int64_t *launches) {
    if (fm_status st = check_problem(p)) return st;
    if (!ms || !launches) return fail(FM_EINVAL, "ms and launches must not be NULL");
    if (pass < 0 || pass >= FM_NUM_PASSES) return fail(FM_EINVAL, "unknown pass");
    FM_CUDA(cudaStreamSynchronize(p->s));
    double total = 0.0;
    for (size_t k = 0; k + 1 < p->tev_used[pass]; k += 2) {
        float t = 0.f;
        FM_CUDA(cudaEventElapsedTime(&t, p->tev[pass][k], p->tev[pass][k + 1]));
        total += t;
    }
    *ms = total;
    *launches = (int64_t)(p->tev_used[pass] / 2);
    p->tev_used[pass] = 0;
    return FM_OK;
}

FM_API fm_status fm_kernel_time(fm_problem *p, double *ms, int64_t *launches) {
    return fm_pass_time(p, FM_PASS_STREAM_LOSS, ms, launches);
}

FM_API const char *fm_status_string(fm_status s) {
    switch (s) {
        case FM_OK: return "FM_OK";
        case FM_EINVAL: return "FM_EINVAL";
        case FM_ENOMEM: return "FM_ENOMEM";
        case FM_ECUDA: return "FM_ECUDA";
        case FM_EDEGENERATE: return "FM_EDEGENERATE";
        case FM_ESTATE: return "FM_ESTATE";
    }
    return "FM_UNKNOWN";
}

FM_API const char *fm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
