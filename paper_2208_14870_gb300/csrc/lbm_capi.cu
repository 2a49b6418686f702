// lbm_capi.cu -- the C ABI of include/lbm.h: context lifetime, parameter
// mapping (Table 1), host <-> device transfers and the pseudo-time driver
// (iterate / solve) around the kernels of lbm_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

// Shared with the batched and serving modules: the message lbm_last_error()
// returns on this host thread.
namespace lbm {
int set_last_error(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
}  // namespace lbm

struct lbm_ctx {
    int device = 0;
    int nx = 0, ny = 0, dtype = 0;
    int64_t n = 0, plane = 0;
    lbm_rates rates{};
    bool gen = false;              // non-standard w_12, w_21, w_22
    cudaStream_t stream = nullptr;
    void* pop[2] = {nullptr, nullptr};
    float* car[2] = {nullptr, nullptr};
    void* force = nullptr;         // 2 planes of the storage force type
    void* snap = nullptr;          // residual snapshot: 2 planes of n entries of 8 bytes (ResSnap)
    double* partials = nullptr;    // residual partial sets, kRes doubles each
    int64_t partials_len = 0;      // partial sets the buffer holds
    double* result = nullptr;      // kRes doubles (device)
    unsigned long long* absmax = nullptr;
    unsigned int* bad = nullptr;
    double* pinned = nullptr;      // kRes + 2 doubles (pinned host)
    double* staging = nullptr;     // FP64 device staging for host transfers
    int64_t staging_len = 0;
    bool staged_fields = false;    // staging holds the fields of the current state and force
    int cur = 0;
    int64_t step = 0;
    bool snap_valid = false;
    int64_t snap_step = 0;
    int hexp = 0;                  // F16S: the state is kept in units scaled by 2^hexp (store_f16s)
    int force_exp = 0;             // F16S: the device force is scaled by 2^force_exp
    float hscale = 1.0f, hinv = 1.0f;
    double gmax = 0.0;             // max |g| of the current force
    bool state_zero = true;        // state is the zero state (create / reset)
    int V = 1;
    size_t bytes = 0;
    int64_t nblocks = 0;           // grid of the residual-check launch
    int spl = 1;                   // pseudo-time steps per stream-collide launch (1 to 4)
    int wave = 0;                  // launches of three or four steps: 0 tile kernel, > 0 wavefront
    int host_transfer = LBM_HOST_DIRECT;   // lbm_host_transfer
                                   // kernel with segments of this many rows per block, -1 wavefront
                                   // with the segment chosen per launch (wave_seg)
    int nsm = 0;                   // multiprocessors of the device
    int64_t nblocks2 = 0;          // grid of the two-step check launch
};

namespace {

size_t pop_elem_bytes(int dtype) {
    return dtype == LBM_F64 ? sizeof(double) : dtype == LBM_F32 ? sizeof(float) : sizeof(__half);
}
size_t force_elem_bytes(int dtype) { return dtype == LBM_F64 ? sizeof(double) : sizeof(float); }

StepParams params(const lbm_ctx* c, int src) {
    StepParams a{};
    a.nx = c->nx;
    a.ny = c->ny;
    a.plane = c->plane;
    a.src = c->pop[src];
    a.dst = c->pop[src ^ 1];
    a.csrc = c->car[src];
    a.cdst = c->car[src ^ 1];
    a.gx = c->force;
    a.gy = static_cast<const char*>(c->force) + c->plane * force_elem_bytes(c->dtype);
    a.hscale = c->hscale;
    a.hinv = c->hinv;
    a.snap = c->snap;
    a.partials = c->partials;
    a.counter = nullptr;   // check launches write partials; k_residual_finish combines them
    a.result = c->result;
    return a;
}

template <typename T>
Coef<T> coef(const lbm_rates& r) {
    Coef<T> c;
    // quarter form (exact scaling by 1/4 before the rounding to T)
    c.q11 = T(0.25 * (1.0 - r.w11));
    c.qs = T(0.25 * (1.0 - r.ws));
    c.qd = T(0.25 * (1.0 - r.wd));
    c.qw12t = T(0.25 * (r.w12 * r.theta));
    c.q12 = T(0.25 * (1.0 - r.w12));
    c.qw21t = T(0.25 * (r.w21 * r.theta));
    c.q21 = T(0.25 * (1.0 - r.w21));
    c.q22 = T(0.25 * (1.0 - r.w22));
    c.qtheta = T(0.25 * r.theta);
    c.theta = T(r.theta);
    c.b11 = T(1.0 - 0.5 * r.w11);
    c.bs = T(1.0 - 0.5 * r.ws);
    c.bd = T(1.0 - 0.5 * r.wd);
    return c;
}

// Residual of a check launch whose blocks wrote partials only.
cudaError_t finish_residual_launch(lbm_ctx* c, int64_t grid) {
    k_residual_finish<<<1, kFinishThreads, 0, c->stream>>>(c->partials, grid, c->result);
    return cudaGetLastError();
}

cudaError_t launch_step(lbm_ctx* c, bool check) {
    const StepParams a = params(c, c->cur);
    cudaError_t e;
    switch (c->dtype) {
        case LBM_F64: e = Ops<S_F64>::step(a, coef<double>(c->rates), c->V, c->gen, check, (int)c->nblocks, c->stream); break;
        case LBM_F32: e = Ops<S_F32>::step(a, coef<float>(c->rates), c->V, c->gen, check, (int)c->nblocks, c->stream); break;
        default: e = Ops<S_F16S>::step(a, coef<float>(c->rates), c->V, c->gen, check, (int)c->nblocks, c->stream); break;
    }
    if (e == cudaSuccess && check) e = finish_residual_launch(c, c->nblocks);
    if (e == cudaSuccess) {
        c->cur ^= 1;
        c->step += 1;
        c->staged_fields = false;
    }
    return e;
}

// Two steps in one launch (FP32 or FP16-shifted storage); with check the
// second step is the residual-check step.
cudaError_t launch_step2(lbm_ctx* c, bool check) {
    const StepParams a = params(c, c->cur);
    cudaError_t e = c->dtype == LBM_F32
                        ? step2_f32(a, coef<float>(c->rates), c->gen, check, (int)c->nblocks2, c->stream)
                        : step2_f16s(a, coef<float>(c->rates), c->gen, check, (int)c->nblocks2, c->stream);
    if (e == cudaSuccess && check) e = finish_residual_launch(c, c->nblocks2);
    if (e == cudaSuccess) {
        c->cur ^= 1;
        c->step += 2;
        c->staged_fields = false;
    }
    return e;
}

// Three plain steps in one launch (FP32 or FP16-shifted storage).
cudaError_t launch_step3(lbm_ctx* c) {
    const StepParams a = params(c, c->cur);
    cudaError_t e = c->dtype == LBM_F32
                        ? step3_f32(a, coef<float>(c->rates), c->gen, false, 0, c->stream)
                        : step3_f16s(a, coef<float>(c->rates), c->gen, false, 0, c->stream);
    if (e == cudaSuccess) {
        c->cur ^= 1;
        c->step += 3;
        c->staged_fields = false;
    }
    return e;
}

// Segment rows of a wavefront launch of T steps: the set value, or (-1)
// kWvSegDefault halved, down to 16, while the grid would have fewer than four
// waves of resident blocks (short segments cost 2(T - j) extra rows at level j).
int wave_seg(const lbm_ctx* c, int T) {
    if (c->wave > 0) return c->wave;
    const int minb = c->dtype == LBM_F16S ? (T == 3 ? wv_minb<S_F16S, 3>() : wv_minb<S_F16S, 4>())
                                          : (T == 3 ? wv_minb<S_F32, 3>() : wv_minb<S_F32, 4>());
    const int64_t want = 4LL * (c->nsm > 0 ? c->nsm : 1) * minb;
    int seg = kWvSegDefault;
    while (seg > 16 && (T == 3 ? wave_blocks<3>(c->nx, c->ny, seg) : wave_blocks<4>(c->nx, c->ny, seg)) < want)
        seg /= 2;
    return seg;
}

// T = 3 or 4 plain steps in one launch: the wavefront kernel where it is on
// and fits, else (T = 3) the three-step tile kernel.
cudaError_t launch_multi(lbm_ctx* c, int T) {
    if (!(c->wave != 0 && wave_fits(c->nx, c->ny))) return T == 3 ? launch_step3(c) : cudaErrorInvalidValue;
    const StepParams a = params(c, c->cur);
    const int seg = wave_seg(c, T);
    cudaError_t e = c->dtype == LBM_F32 ? wave_f32(a, coef<float>(c->rates), c->gen, T, false, seg, c->stream)
                                        : wave_f16s(a, coef<float>(c->rates), c->gen, T, false, seg, c->stream);
    if (e == cudaSuccess) {
        c->cur ^= 1;
        c->step += T;
        c->staged_fields = false;
    }
    return e;
}

int ensure_partials(lbm_ctx* c, int64_t sets);

// Four steps on the wavefront schedule whose last step carries the residual
// check (one partial set per block, combined by k_residual_finish).
cudaError_t launch_wave_checked(lbm_ctx* c) {
    const int seg = wave_seg(c, 4);
    const int64_t blocks = wave_blocks<4>(c->nx, c->ny, seg);
    if (ensure_partials(c, blocks) != LBM_OK) return cudaErrorMemoryAllocation;
    const StepParams a = params(c, c->cur);
    cudaError_t e = c->dtype == LBM_F32 ? wave_f32(a, coef<float>(c->rates), c->gen, 4, true, seg, c->stream)
                                        : wave_f16s(a, coef<float>(c->rates), c->gen, 4, true, seg, c->stream);
    if (e == cudaSuccess) e = finish_residual_launch(c, blocks);
    if (e == cudaSuccess) {
        c->cur ^= 1;
        c->step += 4;
        c->staged_fields = false;
    }
    return e;
}

// n plain steps, grouped into launches of c->spl steps (four only on the
// wavefront schedule, else three); a remainder of one step is avoided where
// possible (4 = 2 + 2, 5 = 3 + 2), since a pair of steps costs about as much
// as one step alone.
cudaError_t run_plain(lbm_ctx* c, int64_t n) {
    cudaError_t e = cudaSuccess;
    const bool wave = c->wave != 0 && wave_fits(c->nx, c->ny);
    const int big = c->spl >= 4 && wave ? 4 : (c->spl >= 3 ? 3 : 0);
    if (big) {
        int64_t groups = n / big, r = n % big;
        if (r == 1 && groups >= 1) {
            --groups;
            r += big;
        }
        for (int64_t i = 0; i < groups && e == cudaSuccess; ++i) e = launch_multi(c, big);
        n = r;
        if (big == 4 && n >= 3 && e == cudaSuccess) {
            e = launch_multi(c, 3);
            n -= 3;
        }
    }
    if (c->spl >= 2)
        for (; n >= 2 && e == cudaSuccess; n -= 2) e = launch_step2(c, false);
    for (; n > 0 && e == cudaSuccess; --n) e = launch_step(c, false);
    return e;
}

// to_check - 1 plain steps followed by the residual-check step (the last
// step of the last launch).  On the four-step wavefront schedule the check is
// the last level of a four-step launch; with three steps per launch on tiles
// it rides on a two-step launch (a three-step tile launch with the check
// costs twice a plain one, a two-step launch with the check 1.3 times).
cudaError_t run_window(lbm_ctx* c, int64_t to_check) {
    cudaError_t e;
    if (c->spl >= 4 && to_check >= 4 && c->wave != 0 && wave_fits(c->nx, c->ny)) {
        e = run_plain(c, to_check - 4);
        return e == cudaSuccess ? launch_wave_checked(c) : e;
    }
    if (c->spl >= 2 && to_check >= 2) {
        e = run_plain(c, to_check - 2);
        return e == cudaSuccess ? launch_step2(c, true) : e;
    }
    e = run_plain(c, to_check - 1);
    return e == cudaSuccess ? launch_step(c, true) : e;
}

cudaError_t launch_fields(lbm_ctx* c, const FieldOut& out);
int ensure_staging(lbm_ctx* c, int64_t len);

// The five FP64 field planes of the current state in the staging buffer,
// computed once per state: lbm_get_displacement and lbm_get_stress of the
// same state share one field recovery.
int stage_fields(lbm_ctx* c) {
    if (c->staged_fields) return LBM_OK;
    int rc = ensure_staging(c, 5 * c->n);
    if (rc) return rc;
    CK(launch_fields(c, field_planes(c->staging, c->n)));
    c->staged_fields = true;
    return LBM_OK;
}

cudaError_t launch_fields(lbm_ctx* c, const FieldOut& out) {
    const StepParams a = params(c, c->cur);
    const Coef<double> cd = coef<double>(c->rates);
    switch (c->dtype) {
        case LBM_F64: return Ops<S_F64>::fields(a, cd, c->rates.theta, out, c->stream);
        case LBM_F32: return Ops<S_F32>::fields(a, cd, float(c->rates.theta), out, c->stream);
        default: return Ops<S_F16S>::fields(a, cd, float(c->rates.theta), out, c->stream);
    }
}

int ensure_staging(lbm_ctx* c, int64_t len) {
    c->staged_fields = false;   // every caller overwrites the staging buffer
    if (c->staging_len >= len) return LBM_OK;
    if (c->staging) {
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaFree(c->staging));
        c->bytes -= c->staging_len * sizeof(double);
        c->staging = nullptr;
        c->staging_len = 0;
    }
    CK(cudaMalloc(&c->staging, len * sizeof(double)));
    c->staging_len = len;
    c->bytes += len * sizeof(double);
    return LBM_OK;
}

// A partials buffer of at least `sets` partial sets (grown on demand: a
// wavefront check launch with short segments may have more blocks than the
// tile launches it was sized for).
int ensure_partials(lbm_ctx* c, int64_t sets) {
    if (c->partials_len >= sets) return LBM_OK;
    if (c->partials) {
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaFree(c->partials));
        c->bytes -= c->partials_len * kRes * sizeof(double);
        c->partials = nullptr;
        c->partials_len = 0;
    }
    CK(cudaMalloc((void**)&c->partials, sets * kRes * sizeof(double)));
    c->partials_len = sets;
    c->bytes += sets * kRes * sizeof(double);
    return LBM_OK;
}

int check_ctx(lbm_ctx* c) {
    if (!c) return fail(LBM_ERR_ARG, "null context");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device) CK(cudaSetDevice(c->device));
    return LBM_OK;
}

void free_all(lbm_ctx* c) {
    for (int i = 0; i < 2; ++i) {
        if (c->pop[i]) cudaFree(c->pop[i]);
        if (c->car[i]) cudaFree(c->car[i]);
    }
    if (c->force) cudaFree(c->force);
    if (c->snap) cudaFree(c->snap);
    if (c->partials) cudaFree(c->partials);
    if (c->result) cudaFree(c->result);
    if (c->absmax) cudaFree(c->absmax);
    if (c->bad) cudaFree(c->bad);
    if (c->staging) cudaFree(c->staging);
    if (c->pinned) cudaFreeHost(c->pinned);
}

// FP16-shifted storage: scale exponent from the force (f16s_exponent).
int half_exponent(const lbm_ctx* c, double gmax) { return f16s_exponent(gmax, c->nx, c->ny); }

// Switch the FP16S scale to 2^e.  rescale: the state is non-zero and is
// carried over -- stored deviations and carriers are multiplied by the power
// of two (the residual snapshot, in the old units, is dropped).  The device
// force always follows the scale (sync_force_scale).
int sync_force_scale(lbm_ctx* c);

int set_half_exponent(lbm_ctx* c, int e, bool rescale) {
    if (e != c->hexp) {
        c->staged_fields = false;
        if (rescale) {
            const float factor = std::ldexp(1.0f, e - c->hexp);
            k_rescale_half<<<1024, 256, 0, c->stream>>>(static_cast<__half*>(c->pop[c->cur]),
                                                       8 * c->plane, factor);
            CK(cudaGetLastError());
            k_scale_float<<<1024, 256, 0, c->stream>>>(c->car[c->cur], 2 * c->plane, factor);
            CK(cudaGetLastError());
            c->snap_valid = false;
        }
        c->hexp = e;
        c->hscale = std::ldexp(1.0f, e);
        c->hinv = std::ldexp(1.0f, -e);
    }
    return sync_force_scale(c);
}

// FP16S: bring the FP32 force on the device to the state's scale 2^hexp.
int sync_force_scale(lbm_ctx* c) {
    if (c->dtype != LBM_F16S || c->force_exp == c->hexp) return LBM_OK;
    c->staged_fields = false;
    k_scale_float<<<1024, 256, 0, c->stream>>>(static_cast<float*>(c->force), 2 * c->plane,
                                               std::ldexp(1.0f, c->hexp - c->force_exp));
    CK(cudaGetLastError());
    c->force_exp = c->hexp;
    return LBM_OK;
}

// The force in the storage type from FP64 arrays the device can address
// (device memory, or mapped pinned host memory), in one pass that also finds
// max |g| and non-finite entries; then the FP16 scale.
int set_force_dev(lbm_ctx* c, const double* gx, const double* gy) {
    c->staged_fields = false;
    CK(cudaMemsetAsync(c->absmax, 0, sizeof(unsigned long long), c->stream));
    CK(cudaMemsetAsync(c->bad, 0, sizeof(unsigned int), c->stream));
    if (c->dtype == LBM_F64) {
        double* fx = static_cast<double*>(c->force);
        k_force_ingest<double><<<2048, 256, 0, c->stream>>>(gx, gy, fx, fx + c->plane, c->n, c->absmax, c->bad);
    } else {
        float* fx = static_cast<float*>(c->force);
        k_force_ingest<float><<<2048, 256, 0, c->stream>>>(gx, gy, fx, fx + c->plane, c->n, c->absmax, c->bad);
    }
    CK(cudaGetLastError());
    c->force_exp = 0;   // converted as given
    CK(cudaMemcpyAsync(c->pinned, c->absmax, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->pinned + 1, c->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double gmax;
    std::memcpy(&gmax, c->pinned, sizeof(double));
    unsigned int bad;
    std::memcpy(&bad, c->pinned + 1, sizeof(unsigned int));
    if (bad) return fail(LBM_ERR_ARG, "lbm_set_force: non-finite force");
    c->gmax = gmax;
    if (c->dtype != LBM_F16S) return LBM_OK;
    if (gmax == 0.0) return sync_force_scale(c);
    int e = half_exponent(c, gmax);
    // A non-zero state keeps its scale unless the new force asks for a
    // smaller one: growing the stored values could overflow FP16.
    if (!c->state_zero && e > c->hexp) e = c->hexp;
    return set_half_exponent(c, e, !c->state_zero);
}

// The device address of a host buffer that is pinned and mapped (then the
// device reads or writes it over the host link directly), or null.
const void* mapped_host(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // an unregistered pointer is not an error here
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Reads the residual of the last check; returns r_inf etc. in out[0..4].
int read_residual(lbm_ctx* c, double out[kRes]) {
    CK(cudaMemcpyAsync(c->pinned, c->result, kRes * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < kRes; ++k) out[k] = c->pinned[k];
    return LBM_OK;
}

// Convert the raw reduction [max|du|, max|u|, sum du^2, sum u^2, bad] over a
// window of `steps` steps into [r_inf, r_2, max|u|, ||u||_2, bad]; `unscale`
// takes the norms of u out of the state's scaled units (FP16S: 2^-hexp).
void finish_residual(const double raw[kRes], int64_t steps, double out[kRes], double unscale) {
    const double k = double(steps > 0 ? steps : 1);
    out[0] = raw[1] > 0.0 ? raw[0] / (k * raw[1]) : 0.0;
    out[1] = raw[3] > 0.0 ? std::sqrt(raw[2]) / (k * std::sqrt(raw[3])) : 0.0;
    out[2] = raw[1] * unscale;
    out[3] = std::sqrt(raw[3]) * unscale;
    out[4] = raw[4];
    if (raw[4] != 0.0 || !std::isfinite(raw[0]) || !std::isfinite(raw[1])) {
        out[0] = out[1] = INFINITY;
        out[4] = 1.0;
    }
}

double norm_unscale(const lbm_ctx* c) { return c->dtype == LBM_F16S ? (double)c->hinv : 1.0; }

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

const char* lbm_version(void) { return "gb300-lbm-elastic 0.1 (sm_103a)"; }

int lbm_create_ex(int nx, int ny, double lambda, double mu, int dtype, const lbm_options* opt,
                  lbm_ctx** out) {
    if (!out) return fail(LBM_ERR_ARG, "lbm_create: null output pointer");
    *out = nullptr;
    if (nx < 1 || ny < 1) return fail(LBM_ERR_ARG, "lbm_create: nx and ny must be >= 1");
    if ((int64_t)nx * ny > (int64_t)1 << 34)
        return fail(LBM_ERR_ARG, "lbm_create: lattice larger than 2^34 nodes");
    if (!std::isfinite(lambda) || !std::isfinite(mu))
        return fail(LBM_ERR_ARG, "lbm_create: non-finite Lame parameter");
    if (!(mu > 0.0)) return fail(LBM_ERR_ARG, "lbm_create: mu must be > 0");
    if (!(lambda + mu > 0.0)) return fail(LBM_ERR_ARG, "lbm_create: lambda + mu must be > 0");
    if (dtype != LBM_F64 && dtype != LBM_F32 && dtype != LBM_F16S)
        return fail(LBM_ERR_ARG, "lbm_create: unknown dtype");
    double theta = 1.0 / 3.0, tau12 = 0.5, tau22 = 0.5;
    if (opt) {
        if (opt->theta != 0.0) theta = opt->theta;
        if (opt->tau12 != 0.0) tau12 = opt->tau12;
        if (opt->tau22 != 0.0) tau22 = opt->tau22;
    }
    if (!(theta > 0.0 && theta < 1.0)) return fail(LBM_ERR_ARG, "lbm_create: theta must be in (0, 1)");
    if (!(tau12 > -0.5) || !(tau22 > -0.5) || !std::isfinite(tau12) || !std::isfinite(tau22))
        return fail(LBM_ERR_ARG, "lbm_create: tau12, tau22 must be finite and > -1/2");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_OOM, "lbm_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDevice");
    }
    c->nx = nx;
    c->ny = ny;
    c->dtype = dtype;
    c->n = (int64_t)nx * ny;
    c->plane = round_up(c->n, 128);
    // Table 1 and Eq. relaxation_rate: theta tau_11 = mu, (1-theta)/2 tau_d = mu,
    // (1+theta)/2 tau_s = K = lambda + mu, w = 1/(tau + 1/2).
    const double K = lambda + mu;
    const double tau11 = mu / theta, taud = 2.0 * mu / (1.0 - theta), taus = 2.0 * K / (1.0 + theta);
    c->rates.w11 = 1.0 / (tau11 + 0.5);
    c->rates.ws = 1.0 / (taus + 0.5);
    c->rates.wd = 1.0 / (taud + 0.5);
    c->rates.w12 = 1.0 / (tau12 + 0.5);
    c->rates.w21 = c->rates.w12;
    c->rates.w22 = 1.0 / (tau22 + 0.5);
    c->rates.theta = theta;
    c->gen = !(c->rates.w12 == 1.0 && c->rates.w22 == 1.0);
    if (dtype == LBM_F64) c->V = nx >= 64 ? 2 : 1;
    else {
        const int vmax = dtype == LBM_F16S ? max_vec<S_F16S>() : max_vec<S_F32>();
        c->V = nx >= 32 * vmax ? vmax : 1;
    }
    // residual-check grids: one block per tile up to kMaxCheckBlocks
    c->nblocks = std::min(step_tiles(nx, ny, c->V), kMaxCheckBlocks);
    if (dtype != LBM_F64) {
        c->nblocks2 = std::min(step2_tiles(nx, ny), kMaxCheckBlocks);
        // four steps per launch on the wavefront schedule where it fits, else
        // three or two on tiles
        c->wave = -1;
        if (wave_fits(nx, ny)) c->spl = 4;
        else if (step3_fits(nx, ny)) c->spl = 3;
        else if (step2_fits(nx, ny)) c->spl = 2;
    }

    const size_t pb = pop_elem_bytes(dtype) * 8 * c->plane;
    const size_t fb = force_elem_bytes(dtype) * 2 * c->plane;
    const size_t cb = sizeof(float) * 2 * c->plane;
    auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, bytes);
        if (r == cudaSuccess) c->bytes += bytes;
        return r;
    };
    e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = alloc(&c->pop[i], pb);
        if (e == cudaSuccess && dtype == LBM_F16S) e = alloc((void**)&c->car[i], cb);
    }
    if (e == cudaSuccess) e = alloc(&c->force, fb);
    // FP64: two planes of doubles; FP32 / FP16S: two planes of (hi, lo) FP32 pairs
    const size_t snap_bytes = 16 * (size_t)c->n;
    if (e == cudaSuccess) e = alloc(&c->snap, snap_bytes);
    c->partials_len = std::max(c->nblocks, c->nblocks2);
    if (dtype != LBM_F64 && wave_fits(nx, ny))
        c->partials_len = std::max(c->partials_len, wave_blocks<4>(nx, ny, wave_seg(c, 4)));
    if (e == cudaSuccess) e = alloc((void**)&c->partials, sizeof(double) * kRes * c->partials_len);
    if (e == cudaSuccess) e = alloc((void**)&c->result, sizeof(double) * kRes);
    if (e == cudaSuccess) e = alloc((void**)&c->absmax, sizeof(unsigned long long));
    if (e == cudaSuccess) e = alloc((void**)&c->bad, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->pinned, sizeof(double) * (kRes + 2));
    if (e == cudaSuccess) e = cudaMemset(c->pop[0], 0, pb);
    if (e == cudaSuccess) e = cudaMemset(c->pop[1], 0, pb);
    if (e == cudaSuccess && dtype == LBM_F16S) e = cudaMemset(c->car[0], 0, cb);
    if (e == cudaSuccess && dtype == LBM_F16S) e = cudaMemset(c->car[1], 0, cb);
    if (e == cudaSuccess) e = cudaMemset(c->force, 0, fb);
    if (e == cudaSuccess) e = cudaMemset(c->snap, 0, snap_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int code = cuda_fail(e, "lbm_create: device allocation");
        free_all(c);
        delete c;
        return code;
    }
    *out = c;
    return LBM_OK;
}

int lbm_create(int nx, int ny, double lambda, double mu, int dtype, lbm_ctx** out) {
    return lbm_create_ex(nx, ny, lambda, mu, dtype, nullptr, out);
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != c->device) cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    if (dev >= 0 && dev != c->device) cudaSetDevice(dev);
    delete c;
}

int lbm_set_steps_per_launch(lbm_ctx* c, int k) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (k < 1 || k > 4) return fail(LBM_ERR_ARG, "lbm_set_steps_per_launch: k must be 1, 2, 3 or 4");
    if (k > 1 && c->dtype == LBM_F64)
        return fail(LBM_ERR_ARG,
                    "lbm_set_steps_per_launch: several steps per launch need FP32 or FP16-shifted storage");
    c->spl = k;
    return LBM_OK;
}

int lbm_get_steps_per_launch(lbm_ctx* c, int* k) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!k) return fail(LBM_ERR_ARG, "lbm_get_steps_per_launch: null pointer");
    *k = c->spl;
    return LBM_OK;
}

int lbm_set_wavefront(lbm_ctx* c, int rows) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (rows < -1 || rows > (1 << 20))
        return fail(LBM_ERR_ARG, "lbm_set_wavefront: rows must be -1 (automatic), 0 (off) or in [1, 2^20]");
    if (rows != 0 && c->dtype == LBM_F64)
        return fail(LBM_ERR_ARG, "lbm_set_wavefront: the wavefront kernel needs FP32 or FP16-shifted storage");
    c->wave = rows;
    return LBM_OK;
}

int lbm_get_wavefront(lbm_ctx* c, int* rows) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!rows) return fail(LBM_ERR_ARG, "lbm_get_wavefront: null pointer");
    *rows = c->wave;
    return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    c->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm_set_host_transfer(lbm_ctx* c, int mode) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (mode != LBM_HOST_DIRECT && mode != LBM_HOST_COPY)
        return fail(LBM_ERR_ARG, "lbm_set_host_transfer: mode must be LBM_HOST_DIRECT or LBM_HOST_COPY");
    c->host_transfer = mode;
    return LBM_OK;
}

int lbm_get_host_transfer(lbm_ctx* c, int* mode) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!mode) return fail(LBM_ERR_ARG, "lbm_get_host_transfer: null pointer");
    *mode = c->host_transfer;
    return LBM_OK;
}

int lbm_set_force(lbm_ctx* c, const double* gx, const double* gy) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!gx || !gy) return fail(LBM_ERR_ARG, "lbm_set_force: null pointer");
    // pinned, mapped host arrays: read by the conversion kernel directly
    // (LBM_HOST_DIRECT), else copied into device staging
    const bool direct = c->host_transfer == LBM_HOST_DIRECT;
    const void* mx = direct ? mapped_host(gx) : nullptr;
    const void* my = direct ? mapped_host(gy) : nullptr;
    if (mx && my) return set_force_dev(c, static_cast<const double*>(mx), static_cast<const double*>(my));
    rc = ensure_staging(c, 2 * c->n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->staging, gx, c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->staging + c->n, gy, c->n * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    return set_force_dev(c, c->staging, c->staging + c->n);
}

int lbm_set_force_corrected(lbm_ctx* c, const double* gx, const double* gy, const double* d) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!gx || !gy || !d) return fail(LBM_ERR_ARG, "lbm_set_force_corrected: null pointer");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(d[i])) return fail(LBM_ERR_ARG, "lbm_set_force_corrected: non-finite D");
    rc = ensure_staging(c, 4 * c->n);
    if (rc) return rc;
    double* in = c->staging;
    double* out = c->staging + 2 * c->n;
    CK(cudaMemcpyAsync(in, gx, c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(in + c->n, gy, c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    k_force_correct<<<1024, 256, 0, c->stream>>>(in, in + c->n, out, out + c->n, c->nx, c->ny, d[0],
                                                 d[1], d[2]);
    CK(cudaGetLastError());
    return set_force_dev(c, out, out + c->n);
}

namespace {

// Appendix B (tau_21 = tau_12): as printed, or (scheme) with the three
// misprints read so that the constants are those of the scheme's exact
// discrete leading error: C2's E^3 term over 8 theta (1 - theta^2)(1 - nu^2)^3
// (printed without theta), and the E terms of D1 and D2 over (1 - theta^2)
// (1 - nu^2) and 2 (1 - theta^2)(1 - nu^2) (printed with (1 - nu^2)^2).
int error_constants(const char* name, double E, double nu, double theta, double tau12, double tau22,
                    bool scheme, double* out) {
    if (!out) return fail(LBM_ERR_ARG, std::string(name) + ": null output");
    if (theta == 0.0) theta = 1.0 / 3.0;
    if (tau12 == 0.0) tau12 = 0.5;
    if (tau22 == 0.0) tau22 = 0.5;
    if (!(E > 0.0) || !(nu > -1.0 && nu < 1.0) || !(theta > 0.0 && theta < 1.0))
        return fail(LBM_ERR_ARG, std::string(name) + ": need E > 0, -1 < nu < 1, 0 < theta < 1");
    const double th = theta, t12 = tau12, t21 = tau12, t22 = tau22;
    const double c = 1.0 - th * th, d = 1.0 - nu * nu, E2 = E * E, E3 = E2 * E;
    const double q = th * th * (1.0 + nu) + nu - 2.0 * th - 1.0;
    out[0] = (nu * nu - 2.0 * th * nu + 1.0) / (c * d * d * d) * E3 +
             th * (nu - th) * t12 / (c * d * d) * E2 +
             (-1.0 + th * th + 12.0 * th * (th - nu) * t12 * t22) / (12.0 * c * d) * E;
    out[1] = ((1.0 - nu) * (1.0 - nu) * (1.0 - nu) + 4.0 * th * (nu * nu * nu - nu * nu + 3.0 * nu + 1.0) +
              th * th * (5.0 * nu * nu * nu - 15.0 * nu * nu - nu - 5.0)) /
                 ((scheme ? 8.0 * th : 8.0) * c * d * d * d) * E3 +
             (2.0 * th * ((1.0 - nu) * nu + th * th * (1.0 + nu) - th * (1.0 + nu * nu)) * t12 +
              (1.0 - th) * (1.0 - nu) * (1.0 + 2.0 * th - nu - th * th * (1.0 + nu)) * t21) /
                 (-4.0 * th * c * d * d) * E2 +
             ((2.0 * th * th - 3.0 * th + 1.0) * (1.0 + 3.0 * th * (1.0 - nu) - 5.0 * nu) +
              24.0 * th * (th - nu) * t12 * t22) / (24.0 * c * d) * E;
    out[2] = ((1.0 - nu) * (1.0 - nu) * (3.0 + nu) + 4.0 * th * (-nu * nu * nu + 3.0 * nu * nu + nu + 1.0) -
              th * th * (5.0 * nu * nu * nu - 3.0 * nu * nu + 7.0 * nu + 7.0)) / (8.0 * th * c * d * d * d) * E3 +
             (-2.0 * (1.0 - th) * th * (nu - 2.0 * th - 1.0) * (1.0 - nu) * t12 -
              ((1.0 + th) * (1.0 - nu) * (1.0 - nu) + th * th * th * (1.0 + nu) * (1.0 + nu) +
               th * th * (nu * nu - 2.0 * nu - 3.0)) * t21) / (4.0 * th * c * d * d) * E2 +
             ((1.0 - th) * (1.0 - nu - th * (1.0 + nu) - 2.0 * th * th * (2.0 + nu)) -
              4.0 * c * (1.0 - nu) * t12 * t22 + 4.0 * q * t21 * t22) / (8.0 * c * d) * E +
             th * t22 / 4.0;
    out[3] = (16.0 * th * nu + (1.0 - nu) * (1.0 - nu) * (3.0 + nu) -
              th * th * (nu * nu * nu + 9.0 * nu * nu - 5.0 * nu + 11.0)) / (8.0 * th * c * d * d * d) * E3 +
             (c * (1.0 - nu) * (th * nu + nu + th - 1.0) * t12 - 2.0 * th * q * t21) / (4.0 * th * c * d * d) * E2 +
             (c * (2.0 * (2.0 - nu) - 3.0 * th * (5.0 + nu)) - 12.0 * c * (1.0 - nu) * t12 * t22 +
              12.0 * q * t21 * t22) / (24.0 * c * d) * E +
             th * t22 / 4.0;
    out[4] = E3 / (8.0 * th * (1.0 + nu) * (1.0 + nu) * (1.0 + nu)) -
             (1.0 - th) * t12 / (4.0 * th * (1.0 + nu) * (1.0 + nu)) * E2 - (3.0 * th - 2.0) / (24.0 * (1.0 + nu)) * E;
    const double dE = scheme ? d : d * d;   // denominator of the E terms of D1, D2 (besides 1 - theta^2)
    out[5] = (nu * nu - 2.0 * th * nu + 1.0) / (c * d * d) * E2 + th * (nu - th) * t12 / (c * dE) * E - 0.25;
    out[6] = ((1.0 - nu) * (1.0 - nu) + 8.0 * th * nu - th * th * (5.0 * nu * nu - 2.0 * nu + 5.0)) /
                 (4.0 * th * c * d * d) * E2 -
             q * t21 / (2.0 * c * dE) * E - th / 2.0;
    out[7] = E2 / (4.0 * th * (1.0 + nu) * (1.0 + nu)) + t12 / (2.0 * (1.0 + nu)) * E - th / 4.0;
    return LBM_OK;
}

}  // namespace

int lbm_error_constants(double E, double nu, double theta, double tau12, double tau22, double* out) {
    return error_constants("lbm_error_constants", E, nu, theta, tau12, tau22, false, out);
}

int lbm_error_constants_scheme(double E, double nu, double theta, double tau12, double tau22, double* out) {
    return error_constants("lbm_error_constants_scheme", E, nu, theta, tau12, tau22, true, out);
}

int lbm_fourth_order_taus(double E, double nu, double theta, double* tau12, double* tau22) {
    if (!tau12 || !tau22) return fail(LBM_ERR_ARG, "lbm_fourth_order_taus: null output");
    if (theta == 0.0) theta = 1.0 / 3.0;
    if (!(E > 0.0) || !(nu > -1.0 && nu < 1.0) || !(theta > 0.0 && theta < 1.0) || nu == theta)
        return fail(LBM_ERR_ARG, "lbm_fourth_order_taus: need E > 0, -1 < nu < 1, 0 < theta < 1, nu != theta");
    // shear modulus (2D relations) and tau_11 of Table 1 (theta tau_11 = mu)
    const double th = theta, mu = E / (2.0 * (1.0 + nu));
    const double t11 = mu / th;
    // Appendix C's tau_12 = tau_21: zeroes C5
    const double t12 = (2.0 - 3.0 * th + 12.0 * th * t11 * t11) / (12.0 * (1.0 - th) * t11);
    // tau_22 from C1 = 0 (C1 of Appendix B, linear in tau_22)
    const double c = 1.0 - th * th, d = 1.0 - nu * nu;
    const double a3 = (nu * nu - 2.0 * th * nu + 1.0) / (c * d * d * d);
    const double a2 = th * (nu - th) / (c * d * d);
    const double t22 = (1.0 - th * th - 12.0 * c * d * (a3 * E * E + a2 * t12 * E)) / (12.0 * th * (th - nu) * t12);
    if (!std::isfinite(t12) || !std::isfinite(t22))
        return fail(LBM_ERR_ARG, "lbm_fourth_order_taus: no finite relaxation times for these parameters");
    *tau12 = t12;
    *tau22 = t22;
    return LBM_OK;
}

int lbm_set_force_device(lbm_ctx* c, const double* gx, const double* gy) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!gx || !gy) return fail(LBM_ERR_ARG, "lbm_set_force_device: null pointer");
    return set_force_dev(c, gx, gy);
}

int lbm_reset(lbm_ctx* c) {
    int rc = check_ctx(c);
    if (rc) return rc;
    CK(cudaMemsetAsync(c->pop[c->cur], 0, pop_elem_bytes(c->dtype) * 8 * c->plane, c->stream));
    if (c->dtype == LBM_F16S)
        CK(cudaMemsetAsync(c->car[c->cur], 0, sizeof(float) * 2 * c->plane, c->stream));
    c->step = 0;
    c->snap_valid = false;
    c->state_zero = true;
    c->staged_fields = false;
    if (c->dtype == LBM_F16S && c->gmax > 0.0) {
        rc = set_half_exponent(c, half_exponent(c, c->gmax), false);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_iterate(lbm_ctx* c, int64_t n) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n < 0) return fail(LBM_ERR_ARG, "lbm_iterate: n must be >= 0");
    if (n > 0) c->state_zero = false;
    cudaError_t e = run_plain(c, n);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_iterate: step launch");
    return LBM_OK;
}

int lbm_iterate_checked(lbm_ctx* c, int64_t n, int check_every, double* out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n < 0 || check_every < 1) return fail(LBM_ERR_ARG, "lbm_iterate_checked: bad n or check_every");
    if (n > 0) c->state_zero = false;
    int64_t last_window = 0;
    bool any = false;
    // a check on every step whose index + 1 is a multiple of check_every
    for (int64_t left = n; left > 0;) {
        const int64_t to_check = check_every - (c->step % check_every);
        if (to_check > left) {
            cudaError_t e = run_plain(c, left);
            if (e != cudaSuccess) return cuda_fail(e, "lbm_iterate_checked: step launch");
            break;
        }
        cudaError_t e = run_window(c, to_check);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_iterate_checked: step launch");
        left -= to_check;
        last_window = c->snap_valid ? c->step - c->snap_step : 0;
        any = c->snap_valid;
        c->snap_valid = true;
        c->snap_step = c->step;
    }
    if (out) {
        double raw[kRes];
        rc = read_residual(c, raw);
        if (rc) return rc;
        if (any) finish_residual(raw, last_window, out, norm_unscale(c));
        else {
            finish_residual(raw, 1, out, norm_unscale(c));
            out[0] = out[1] = INFINITY;
        }
    }
    return LBM_OK;
}

int lbm_solve(lbm_ctx* c, double tol, int64_t max_iters, int check_every, int64_t* iters_out,
              double* residual_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!(tol >= 0.0) || max_iters < 0 || check_every < 1)
        return fail(LBM_ERR_ARG, "lbm_solve: bad tol, max_iters or check_every");
    if (max_iters > 0) c->state_zero = false;
    // windows long enough that the storage's rounding jitter stays below tol,
    // stretched while the residual stagnates (adapt_period)
    const int k = check_every;
    int period = check_period(c->dtype, tol, k, std::min(c->nx, c->ny));
    check_every = k * period;
    int64_t done = 0;
    double r = INFINITY, r_prev = INFINITY;
    int status = LBM_ERR_NOT_CONVERGED;
    while (done < max_iters) {
        const int64_t to_check = check_every - (c->step % check_every);
        if (done + to_check > max_iters) {
            rc = lbm_iterate(c, max_iters - done);
            if (rc) return rc;
            done = max_iters;
            break;
        }
        cudaError_t e = run_window(c, to_check);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_solve: step launch");
        done += to_check;
        double raw[kRes], res[kRes];
        rc = read_residual(c, raw);
        if (rc) return rc;
        const bool had = c->snap_valid;
        const int64_t window = c->step - c->snap_step;
        c->snap_valid = true;
        c->snap_step = c->step;
        finish_residual(raw, window, res, norm_unscale(c));
        if (res[4] != 0.0) {
            status = LBM_ERR_DIVERGED;
            r = INFINITY;
            break;
        }
        if (!had) continue;
        r = res[0];
        if (r < tol) {
            status = LBM_OK;
            break;
        }
        period = adapt_period(period, r, r_prev);
        check_every = k * period;
        r_prev = r;
    }
    if (iters_out) *iters_out = done;
    if (residual_out) *residual_out = r;
    if (status == LBM_ERR_DIVERGED) return fail(status, "lbm_solve: non-finite displacement (diverged)");
    if (status == LBM_ERR_NOT_CONVERGED) return fail(status, "lbm_solve: max_iters reached above tolerance");
    return LBM_OK;
}

int lbm_get_fields_device(lbm_ctx* c, double* out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!out) return fail(LBM_ERR_ARG, "lbm_get_fields_device: null pointer");
    CK(launch_fields(c, field_planes(out, c->n)));
    return LBM_OK;
}

namespace {

// Host field getters: into pinned, mapped host arrays the recovery kernel
// writes directly (only the requested fields; LBM_HOST_DIRECT); other host
// arrays receive copies of the fields staged once per state.
int get_fields_host(lbm_ctx* c, int first, int count, double* const* dst) {
    FieldOut o{};
    bool mapped = c->host_transfer == LBM_HOST_DIRECT;
    for (int k = 0; k < count && mapped; ++k) {
        o.p[first + k] = static_cast<double*>(const_cast<void*>(mapped_host(dst[k])));
        mapped = o.p[first + k] != nullptr;
    }
    if (mapped) {
        CK(launch_fields(c, o));
        CK(cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    int rc = stage_fields(c);
    if (rc) return rc;
    for (int k = 0; k < count; ++k)
        CK(cudaMemcpyAsync(dst[k], c->staging + (first + k) * c->n, c->n * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // namespace

int lbm_get_displacement(lbm_ctx* c, double* ux, double* uy) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!ux || !uy) return fail(LBM_ERR_ARG, "lbm_get_displacement: null pointer");
    double* d[2] = {ux, uy};
    return get_fields_host(c, 0, 2, d);
}

int lbm_get_stress(lbm_ctx* c, double* sxx, double* syy, double* sxy) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!sxx || !syy || !sxy) return fail(LBM_ERR_ARG, "lbm_get_stress: null pointer");
    double* d[3] = {sxx, syy, sxy};
    return get_fields_host(c, 2, 3, d);
}

int lbm_get_populations(lbm_ctx* c, double* f) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!f) return fail(LBM_ERR_ARG, "lbm_get_populations: null pointer");
    rc = ensure_staging(c, 8 * c->n);
    if (rc) return rc;
    const StepParams a = params(c, c->cur);
    cudaError_t e;
    switch (c->dtype) {
        case LBM_F64: e = Ops<S_F64>::export_pop(a, c->rates.theta, c->staging, c->stream); break;
        case LBM_F32: e = Ops<S_F32>::export_pop(a, float(c->rates.theta), c->staging, c->stream); break;
        default: e = Ops<S_F16S>::export_pop(a, float(c->rates.theta), c->staging, c->stream); break;
    }
    CK(e);
    CK(cudaMemcpyAsync(f, c->staging, 8 * c->n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!f) return fail(LBM_ERR_ARG, "lbm_set_populations: null pointer");
    double fmax_abs = 0.0;
    for (int64_t i = 0; i < 8 * c->n; ++i) {
        if (!std::isfinite(f[i])) return fail(LBM_ERR_ARG, "lbm_set_populations: non-finite value");
        fmax_abs = std::fmax(fmax_abs, std::fabs(f[i]));
    }
    if (c->dtype == LBM_F16S && fmax_abs > 0.0) {
        // deviations are bounded by a few times max|f|; keep them below 2^12
        int e = 10 - (int)std::ceil(std::log2(fmax_abs));
        if (c->gmax > 0.0 && half_exponent(c, c->gmax) < e) e = half_exponent(c, c->gmax);
        if (e > 60) e = 60;
        if (e < -60) e = -60;
        rc = set_half_exponent(c, e, false);
        if (rc) return rc;
    }
    rc = ensure_staging(c, 8 * c->n);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->staging, f, 8 * c->n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const StepParams a = params(c, c->cur ^ 1);  // dst = current buffer
    cudaError_t e;
    switch (c->dtype) {
        case LBM_F64: e = Ops<S_F64>::import_pop(a, c->rates.theta, c->staging, c->stream); break;
        case LBM_F32: e = Ops<S_F32>::import_pop(a, float(c->rates.theta), c->staging, c->stream); break;
        default: e = Ops<S_F16S>::import_pop(a, float(c->rates.theta), c->staging, c->stream); break;
    }
    CK(e);
    CK(cudaStreamSynchronize(c->stream));
    c->step = 0;
    c->snap_valid = false;
    c->state_zero = false;
    return LBM_OK;
}

int lbm_get_step(lbm_ctx* c, int64_t* step) {
    if (!c || !step) return fail(LBM_ERR_ARG, "lbm_get_step: null pointer");
    *step = c->step;
    return LBM_OK;
}

int lbm_get_rates(lbm_ctx* c, lbm_rates* out) {
    if (!c || !out) return fail(LBM_ERR_ARG, "lbm_get_rates: null pointer");
    *out = c->rates;
    return LBM_OK;
}

int lbm_get_device_bytes(lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(LBM_ERR_ARG, "lbm_get_device_bytes: null pointer");
    *bytes = c->bytes;
    return LBM_OK;
}

}  // extern "C"
