// lbm_engine.cu -- host side of the packed lattice arena (lbm_engine.cuh).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <sys/stat.h>

#include "../../include/lbm.h"
#include "lbm_engine.cuh"

static_assert(lbm::kTileTwoStep == LBM_TILE_TWO_STEP, "tile code of two-step tiles");
static_assert(lbm::kTileWave == LBM_TILE_WAVE, "tile code of the wavefront chunk");

namespace lbm {

namespace {

int cuerr(cudaError_t e, const char* what, std::string* err) {
    if (err) *err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define ECK(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuerr(e_, #call, err);      \
    } while (0)

int64_t pop_bytes_per_node(int dtype) { return dtype == S_F16S ? 8 * 2 : 8 * 4; }
int64_t car_bytes_per_node(int dtype) { return dtype == S_F16S ? 2 * 4 : 0; }
// force (2 FP32 planes) + residual snapshot (2 planes of (hi, lo) FP32 pairs)
constexpr int64_t kFsBytesPerNode = 2 * 4 + 2 * 8;

}  // namespace

ArenaEngine::~ArenaEngine() {
    if (st_) cudaStreamSynchronize(st_);
    for (auto& g : graph_)
        if (g) cudaGraphExecDestroy(g);
    for (int i = 0; i < 2; ++i) {
        if (pop_[i]) cudaFree(pop_[i]);
        if (car_[i]) cudaFree(car_[i]);
    }
    if (fs_) cudaFree(fs_);
    if (d_probs_) cudaFree(d_probs_);
    if (d_acc_) cudaFree(d_acc_);
    if (d_tiles_) cudaFree(d_tiles_);
    if (d_ntiles_) cudaFree(d_ntiles_);
    if (d_nwide_) cudaFree(d_nwide_);
    if (d_counters_) cudaFree(d_counters_);
    if (d_fields_) cudaFree(d_fields_);
    if (h_acc_) cudaFreeHost(h_acc_);
    if (h_tiles_) cudaFreeHost(h_tiles_);
    if (h_force_) cudaFreeHost(h_force_);
    if (h_fields_) cudaFreeHost(h_fields_);
    if (ev0_) cudaEventDestroy(ev0_);
    if (ev1_) cudaEventDestroy(ev1_);
}

int64_t ArenaEngine::bytes_for(int64_t n) const {
    auto al = [](int64_t b) { return (b + kArenaAlign - 1) / kArenaAlign * kArenaAlign; };
    return 2 * al(pop_bytes_per_node(dtype_) * n) + 2 * al(car_bytes_per_node(dtype_) * n) +
           al(kFsBytesPerNode * n);
}

int ArenaEngine::init(int dtype, int64_t node_capacity, int max_probs, int check_every,
                      cudaStream_t st, std::string* err) {
    if (dtype != S_F32 && dtype != S_F16S) {
        if (err) *err = "arena: storage must be LBM_F32 or LBM_F16S";
        return LBM_ERR_ARG;
    }
    dtype_ = dtype;
    k_ = check_every;
    st_ = st;
    int dev = 0;
    ECK(cudaGetDevice(&dev));
    ECK(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
    const int64_t slack = (int64_t)max_probs * kArenaAlign;
    const int64_t pb = pop_bytes_per_node(dtype) * node_capacity + slack;
    const int64_t cb = car_bytes_per_node(dtype) * node_capacity + slack;
    const int64_t fb = kFsBytesPerNode * node_capacity + slack;
    for (int i = 0; i < 2; ++i) {
        ECK(cudaMalloc(&pop_[i], pb));
        dev_bytes_ += pb;
        if (dtype == S_F16S) {
            ECK(cudaMalloc(&car_[i], cb));
            dev_bytes_ += cb;
        }
    }
    ECK(cudaMalloc(&fs_, fb));
    dev_bytes_ += fb;
    apop_.reset(pb);
    acar_.reset(dtype == S_F16S ? cb : 0);
    afs_.reset(fb);
    probs_.assign(max_probs, HostProb());
    ECK(cudaMalloc(&d_probs_, sizeof(BatchProb) * max_probs));
    ECK(cudaMalloc(&d_acc_, sizeof(double) * kRes * max_probs));
    ECK(cudaMallocHost(&h_acc_, sizeof(double) * kRes * max_probs));
    ECK(cudaMalloc(&d_ntiles_, sizeof(int)));
    ECK(cudaMemsetAsync(d_ntiles_, 0, sizeof(int), st_));
    ECK(cudaMalloc(&d_nwide_, sizeof(int)));
    ECK(cudaMemsetAsync(d_nwide_, 0, sizeof(int), st_));
    ECK(cudaMalloc(&d_counters_, sizeof(int) * 2 * (k_ / 4 + 1)));
    ECK(cudaEventCreate(&ev0_));
    ECK(cudaEventCreate(&ev1_));
    dev_bytes_ += sizeof(BatchProb) * max_probs + sizeof(double) * kRes * max_probs;
    return LBM_OK;
}

int ArenaEngine::admit(int nx, int ny, double lambda, double mu, const double* gx, const double* gy,
                       double tol, int64_t max_iters, std::string* err) {
    if (nx < 1 || ny < 1 || !gx || !gy || !(mu > 0.0) || !(lambda + mu > 0.0) ||
        !std::isfinite(lambda) || !std::isfinite(mu)) {
        if (err) *err = "admit: bad problem (sizes, moduli or null force)";
        return LBM_ERR_ARG;
    }
    int slot = -1;
    for (int i = 0; i < (int)probs_.size(); ++i)
        if (probs_[i].state == P_FREE) {
            slot = i;
            break;
        }
    if (slot < 0) return -1;
    const int64_t n = (int64_t)nx * ny;
    HostProb p;
    p.pop_bytes = pop_bytes_per_node(dtype_) * n;
    p.car_bytes = car_bytes_per_node(dtype_) * n;
    p.fs_bytes = kFsBytesPerNode * n;
    p.pop_off = apop_.alloc(p.pop_bytes);
    if (p.pop_off < 0) return -1;
    if (dtype_ == S_F16S) {
        p.car_off = acar_.alloc(p.car_bytes);
        if (p.car_off < 0) {
            apop_.release(p.pop_off, p.pop_bytes);
            return -1;
        }
    } else {
        p.car_off = 0;
    }
    p.fs_off = afs_.alloc(p.fs_bytes);
    if (p.fs_off < 0) {
        apop_.release(p.pop_off, p.pop_bytes);
        if (dtype_ == S_F16S) acar_.release(p.car_off, p.car_bytes);
        return -1;
    }
    // a problem that is cheaper on its transpose is solved there: lattice
    // ny x nx, force components exchanged, node (x, y) at x * ny + y
    const bool tr = arena_transpose(nx, ny);
    // force -> FP32 staging (pinned), with the FP16 scale from its maximum
    if (h_force_cap_ < 2 * n) {
        if (h_force_) {
            ECK(cudaStreamSynchronize(st_));
            cudaFreeHost(h_force_);
            h_force_ = nullptr;
        }
        ECK(cudaMallocHost(&h_force_, sizeof(float) * 2 * n));
        h_force_cap_ = 2 * n;
    }
    ECK(cudaStreamSynchronize(st_));  // the staging may still feed a previous copy
    double gmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double a = gx[i], b = gy[i];
        if (!std::isfinite(a) || !std::isfinite(b)) {
            apop_.release(p.pop_off, p.pop_bytes);
            if (dtype_ == S_F16S) acar_.release(p.car_off, p.car_bytes);
            afs_.release(p.fs_off, p.fs_bytes);
            if (err) *err = "admit: non-finite force";
            return LBM_ERR_ARG;
        }
        gmax = std::fmax(gmax, std::fmax(std::fabs(a), std::fabs(b)));
        if (tr) {
            const int64_t t = (i % nx) * ny + i / nx;
            h_force_[t] = (float)b;
            h_force_[n + t] = (float)a;
        } else {
            h_force_[i] = (float)a;
            h_force_[n + i] = (float)b;
        }
    }
    if (tr) std::swap(nx, ny);
    p.hexp = dtype_ == S_F16S ? f16s_exponent(gmax, nx, ny) : 0;
    if (p.hexp != 0) {
        // FP16S keeps its state, the force included, in units scaled by 2^hexp
        // (store_f16s); the power of two is exact
        const float sc = std::ldexp(1.0f, p.hexp);
        for (int64_t i = 0; i < 2 * n; ++i) h_force_[i] *= sc;
    }
    ECK(cudaMemcpyAsync(fs_ + p.fs_off, h_force_, sizeof(float) * 2 * n, cudaMemcpyHostToDevice, st_));
    ECK(cudaMemsetAsync(fs_ + p.fs_off + sizeof(float) * 2 * n, 0, sizeof(float2) * 2 * n, st_));
    ECK(cudaMemsetAsync(pop_[0] + p.pop_off, 0, p.pop_bytes, st_));
    if (dtype_ == S_F16S) ECK(cudaMemsetAsync(car_[0] + p.car_off, 0, p.car_bytes, st_));
    p.parity = 0;
    p.nx = nx;
    p.ny = ny;
    p.tr = tr;
    p.n = n;
    p.lambda = lambda;
    p.mu = mu;
    // Table 1 / Eq. relaxation_rate with theta = 1/3, w_12 = w_21 = w_22 = 1
    const double theta = 1.0 / 3.0, K = lambda + mu;
    p.theta = (float)theta;
    p.qtheta = (float)(0.25 * theta);   // quarter form of collide
    p.q11 = (float)(0.25 * (1.0 - 1.0 / (mu / theta + 0.5)));
    p.qs = (float)(0.25 * (1.0 - 1.0 / (2.0 * K / (1.0 + theta) + 0.5)));
    p.qd = (float)(0.25 * (1.0 - 1.0 / (2.0 * mu / (1.0 - theta) + 0.5)));
    p.tol = tol;
    p.max_iters = max_iters;
    p.period = check_period(dtype_, tol, k_, std::min(nx, ny));
    p.r_prev = INFINITY;
    p.last_check = 0;
    p.state = P_RUNNING;
    probs_[slot] = p;
    ++nrunning_;
    tiles_dirty_ = true;
    desc_dirty_ = true;
    return slot;
}

int64_t ArenaEngine::running_tiles(int V, int seg) const {
    int64_t t = 0;
    for (const auto& p : probs_)
        if (p.state == P_RUNNING) t += arena_tiles(p.nx, p.ny, V, seg);
    return t;
}

int64_t ArenaEngine::running_nodes() const {
    int64_t t = 0;
    for (const auto& p : probs_)
        if (p.state == P_RUNNING) t += p.n;
    return t;
}

int64_t ArenaEngine::resident_bytes() const {
    int64_t b = 0;
    for (const auto& p : probs_)
        if (p.state != P_FREE) b += bytes_for(p.n);
    return b;
}

int ArenaEngine::grid_blocks(int V) const { return arena_occupancy(dtype_, V) * sms_; }

int64_t ArenaEngine::free_nodes_hint() const {
    return apop_.largest_free() / pop_bytes_per_node(dtype_);
}

int ArenaEngine::upload_tiles(int V, std::string* err) {
    if (V == kTileWave) {
        // longest segments that still give four waves of resident blocks
        const int64_t want = 4LL * grid_blocks(V);
        int seg = kArenaWaveSegMax;
        while (seg > 16 && running_tiles(V, seg) < want) seg /= 2;
        if (seg != wave_seg_) desc_dirty_ = true;
        wave_seg_ = seg;
    }
    const int64_t nt = running_tiles(V, wave_seg_);
    if (nt > (int64_t)INT32_MAX) {
        if (err) *err = "arena: too many tiles";
        return LBM_ERR_ARG;
    }
    if (h_tiles_cap_ < nt) {
        if (h_tiles_) {
            ECK(cudaStreamSynchronize(st_));
            cudaFreeHost(h_tiles_);
        }
        h_tiles_cap_ = nt + nt / 4 + 1024;
        ECK(cudaMallocHost(&h_tiles_, sizeof(uint2) * h_tiles_cap_));
    }
    if (tiles_cap_ < nt) {
        if (d_tiles_) {
            ECK(cudaStreamSynchronize(st_));
            cudaFree(d_tiles_);
        }
        tiles_cap_ = nt + nt / 4 + 1024;
        ECK(cudaMalloc(&d_tiles_, sizeof(uint2) * tiles_cap_));
        for (auto& g : graph_)  // the graphs hold the old tile pointer
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    ECK(cudaStreamSynchronize(st_));  // the pinned list may feed a previous copy
    // wavefront chunks list the wide problems' wavefront items first, then the
    // narrow problems' two-step tiles
    int64_t t = 0, nwide = 0;
    for (int pass = (V == kTileWave ? 0 : 1); pass < 2; ++pass) {
        for (int s = 0; s < (int)probs_.size(); ++s) {
            const HostProb& p = probs_[s];
            if (p.state != P_RUNNING) continue;
            if (V == kTileWave && arena_wide(p.nx, p.ny) != (pass == 0)) continue;
            const int64_t m = arena_tiles(p.nx, p.ny, V, wave_seg_);
            for (int64_t i = 0; i < m; ++i) h_tiles_[t++] = make_uint2((unsigned)s, (unsigned)i);
        }
        if (pass == 0) nwide = t;
    }
    static thread_local int nt_host[2];
    nt_host[0] = (int)nt;
    nt_host[1] = (int)nwide;
    if (nt > 0) ECK(cudaMemcpyAsync(d_tiles_, h_tiles_, sizeof(uint2) * nt, cudaMemcpyHostToDevice, st_));
    ECK(cudaMemcpyAsync(d_ntiles_, &nt_host[0], sizeof(int), cudaMemcpyHostToDevice, st_));
    ECK(cudaMemcpyAsync(d_nwide_, &nt_host[1], sizeof(int), cudaMemcpyHostToDevice, st_));
    ECK(cudaStreamSynchronize(st_));
    tiles_V_ = V;
    tiles_dirty_ = false;
    return LBM_OK;
}

BatchArgs ArenaEngine::chunk_args() const {
    BatchArgs a{};
    a.probs = d_probs_;
    a.tiles = d_tiles_;
    a.ntiles = d_ntiles_;
    a.nwide = d_nwide_;
    a.counters = d_counters_;
    a.pop0 = pop_[0];
    a.pop1 = pop_[1];
    a.car0 = car_[0];
    a.car1 = car_[1];
    a.fs = fs_;
    a.acc = d_acc_;
    a.nsteps = k_;
    return a;
}

int ArenaEngine::ensure_graph(int V, std::string* err) {
    if (graph_[V] || graph_failed_[V]) return LBM_OK;
    const BatchArgs a = chunk_args();
    const int grid = grid_blocks(V);
    if (grid < 1) {
        if (err) *err = "arena: chunk kernel cannot be resident";
        return LBM_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(d_acc_, 0, sizeof(double) * kRes * probs_.size(), st_);
        if (V == kTileWave) cudaMemsetAsync(d_counters_, 0, sizeof(int) * 2 * (k_ / 4), st_);
        launch_arena_chunk(dtype_, V, a, grid, st_);
        cudaMemcpyAsync(h_acc_, d_acc_, sizeof(double) * kRes * probs_.size(), cudaMemcpyDeviceToHost, st_);
        e = cudaStreamEndCapture(st_, &g);
    }
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&graph_[V], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear; fall back to direct launches
        graph_[V] = nullptr;
        graph_failed_[V] = true;
    }
    return LBM_OK;
}

int ArenaEngine::run_chunk(int V, float* device_ms, std::string* err) {
    if (V != 1 && V != 2 && V != 4 && !(V == kTileTwoStep && k_ % 2 == 0) && !(V == kTileWave && k_ % 4 == 0)) {
        if (err) *err = "arena: tile code must be 1, 2 or 4 warps of 32, two-step tiles with an even chunk, "
                        "or the wavefront chunk with a chunk of a multiple of 4 steps";
        return LBM_ERR_ARG;
    }
    if (device_ms) *device_ms = 0.0f;
    if (nrunning_ == 0) return LBM_OK;
    if (tiles_dirty_ || tiles_V_ != V) {
        int rc = upload_tiles(V, err);
        if (rc) return rc;
    }
    for (auto& p : probs_) {
        if (p.state != P_RUNNING) continue;
        const bool now = ((p.steps + k_) % ((int64_t)k_ * p.period)) == 0;
        if (now != p.check_now) {
            p.check_now = now;
            desc_dirty_ = true;
        }
    }
    if (desc_dirty_) {
        std::vector<BatchProb> d(probs_.size());
        for (size_t i = 0; i < probs_.size(); ++i) {
            const HostProb& p = probs_[i];
            BatchProb& b = d[i];
            b.pop_off = p.pop_off;
            b.car_off = p.car_off;
            b.fs_off = p.fs_off;
            b.nx = p.nx;
            b.ny = p.ny;
            b.check = p.check_now ? 1 : 0;
            b.dtype = dtype_;
            b.parity = p.parity;
            b.seg = wave_seg_;
            b.q11 = p.q11;
            b.qs = p.qs;
            b.qd = p.qd;
            b.qtheta = p.qtheta;
            b.theta = p.theta;
            b.hscale = std::ldexp(1.0f, p.hexp);
            b.hinv = std::ldexp(1.0f, -p.hexp);
        }
        ECK(cudaMemcpyAsync(d_probs_, d.data(), sizeof(BatchProb) * d.size(), cudaMemcpyHostToDevice, st_));
        ECK(cudaStreamSynchronize(st_));
        desc_dirty_ = false;
    }
    int rc = ensure_graph(V, err);
    if (rc) return rc;
    ECK(cudaEventRecord(ev0_, st_));
    if (graph_[V]) {
        ECK(cudaGraphLaunch(graph_[V], st_));
    } else {
        const BatchArgs a = chunk_args();
        ECK(cudaMemsetAsync(d_acc_, 0, sizeof(double) * kRes * probs_.size(), st_));
        if (V == kTileWave) ECK(cudaMemsetAsync(d_counters_, 0, sizeof(int) * 2 * (k_ / 4), st_));
        ECK(launch_arena_chunk(dtype_, V, a, grid_blocks(V), st_));
        ECK(cudaMemcpyAsync(h_acc_, d_acc_, sizeof(double) * kRes * probs_.size(), cudaMemcpyDeviceToHost, st_));
    }
    ECK(cudaEventRecord(ev1_, st_));
    ECK(cudaStreamSynchronize(st_));
    if (device_ms) ECK(cudaEventElapsedTime(device_ms, ev0_, ev1_));
    for (int s = 0; s < (int)probs_.size(); ++s) {
        HostProb& p = probs_[s];
        if (p.state != P_RUNNING) continue;
        p.steps += k_;
        p.lups += p.n * k_;
        // the buffers swap once per launch-level step: k steps, k/2 pairs, or
        // (wavefront chunk) k/4 passes of a wide problem, k/2 pairs of a narrow one
        const int64_t swaps = V == kTileWave ? (arena_wide(p.nx, p.ny) ? k_ / 4 : k_ / 2)
                                             : (V == kTileTwoStep ? k_ / 2 : k_);
        if (swaps & 1) {
            p.parity ^= 1;
            desc_dirty_ = true;
        }
        const double* raw = h_acc_ + (int64_t)s * kRes;
        bool done = false;
        if (!p.check_now) {
            // no residual this chunk
        } else if (raw[4] != 0.0 || !std::isfinite(raw[0]) || !std::isfinite(raw[1])) {
            p.status = LBM_ERR_DIVERGED;
            p.residual = INFINITY;
            done = true;
        } else if (!p.snap_valid) {
            p.snap_valid = true;
            p.residual = INFINITY;
            p.last_check = p.steps;
        } else {
            const double window = (double)(p.steps - p.last_check);
            p.last_check = p.steps;
            p.residual = raw[1] > 0.0 ? raw[0] / (window * raw[1]) : 0.0;
            if (p.residual < p.tol) {
                p.status = LBM_OK;
                done = true;
            } else {
                p.period = adapt_period(p.period, p.residual, p.r_prev);
                p.r_prev = p.residual;
            }
        }
        if (!done && p.steps >= p.max_iters) {
            p.status = LBM_ERR_NOT_CONVERGED;
            done = true;
        }
        if (done) {
            p.state = P_DONE;
            --nrunning_;
            tiles_dirty_ = true;
        }
    }
    return LBM_OK;
}

// FP64 fields of problem `slot` into device memory dst (5 planes of n).
cudaError_t ArenaEngine::launch_fields(int slot, double* dst) {
    const HostProb& p = probs_[slot];
    StepParams a{};
    a.nx = p.nx;
    a.ny = p.ny;
    a.plane = p.n;
    a.src = pop_[p.parity] + p.pop_off;
    a.dst = pop_[p.parity ^ 1] + p.pop_off;
    if (dtype_ == S_F16S) {
        a.csrc = reinterpret_cast<const float*>(car_[p.parity] + p.car_off);
        a.cdst = reinterpret_cast<float*>(car_[p.parity ^ 1] + p.car_off);
        a.hscale = std::ldexp(1.0f, p.hexp);
        a.hinv = std::ldexp(1.0f, -p.hexp);
    }
    float* fsb = reinterpret_cast<float*>(fs_ + p.fs_off);
    a.gx = fsb;
    a.gy = fsb + p.n;
    a.snap = fsb + 2 * p.n;
    const double theta = 1.0 / 3.0, K = p.lambda + p.mu;
    const double w11 = 1.0 / (p.mu / theta + 0.5), ws = 1.0 / (2.0 * K / (1.0 + theta) + 0.5),
                 wd = 1.0 / (2.0 * p.mu / (1.0 - theta) + 0.5);
    Coef<double> c{};
    c.b11 = 1.0 - 0.5 * w11;
    c.bs = 1.0 - 0.5 * ws;
    c.bd = 1.0 - 0.5 * wd;
    c.theta = theta;
    FieldOut o = field_planes(dst, p.n);
    if (p.tr) {
        // back to the caller's lattice: u_x <-> u_y, sigma_xx <-> sigma_yy,
        // node (x, y) of the transpose at x * ny + y
        std::swap(o.p[0], o.p[1]);
        std::swap(o.p[2], o.p[3]);
        o.tr = 1;
    }
    return dtype_ == S_F16S ? Ops<S_F16S>::fields(a, c, (float)theta, o, st_)
                            : Ops<S_F32>::fields(a, c, (float)theta, o, st_);
}

int ArenaEngine::ensure_fields_buffer(int64_t len, std::string* err) {
    if (d_fields_cap_ >= len) return LBM_OK;
    if (d_fields_) {
        ECK(cudaStreamSynchronize(st_));
        cudaFree(d_fields_);
        d_fields_ = nullptr;
        d_fields_cap_ = 0;
    }
    ECK(cudaMalloc(&d_fields_, sizeof(double) * len));
    d_fields_cap_ = len;
    return LBM_OK;
}

int ArenaEngine::recover(int slot, double* ux, double* uy, double* sxx, double* syy, double* sxy,
                         std::string* err) {
    const HostProb& p = probs_[slot];
    if (p.state == P_FREE) {
        if (err) *err = "recover: empty slot";
        return LBM_ERR_STATE;
    }
    int rc = ensure_fields_buffer(5 * p.n, err);
    if (rc) return rc;
    ECK(launch_fields(slot, d_fields_));
    double* outs[5] = {ux, uy, sxx, syy, sxy};
    for (int i = 0; i < 5; ++i)
        if (outs[i])
            ECK(cudaMemcpyAsync(outs[i], d_fields_ + i * p.n, sizeof(double) * p.n,
                                cudaMemcpyDeviceToHost, st_));
    ECK(cudaStreamSynchronize(st_));
    return LBM_OK;
}

int ArenaEngine::recover_many(int count, const int* slots, double* const* outs, std::string* err) {
    // Problems are packed into blocks of kRecoverBlock doubles: one field
    // launch per problem into a device block, one copy of the block into a
    // pinned host block, one synchronisation, then host copies into the
    // callers' arrays.  A problem larger than a block goes alone.
    constexpr int64_t kRecoverBlock = int64_t(4) << 20;   // 32 MB of FP64
    for (int i = 0; i < count; ++i)
        if (probs_[slots[i]].state == P_FREE) {
            if (err) *err = "recover: empty slot";
            return LBM_ERR_STATE;
        }
    int rc = ensure_fields_buffer(kRecoverBlock, err);
    if (rc) return rc;
    if (!h_fields_) {
        ECK(cudaMallocHost(&h_fields_, sizeof(double) * kRecoverBlock));
    }
    for (int i = 0; i < count;) {
        if (5 * probs_[slots[i]].n > kRecoverBlock) {
            double* const* o = outs + 5 * (int64_t)i;
            rc = recover(slots[i], o[0], o[1], o[2], o[3], o[4], err);
            if (rc) return rc;
            ++i;
            continue;
        }
        int j = i;
        int64_t used = 0;
        for (; j < count && 5 * probs_[slots[j]].n <= kRecoverBlock - used; ++j) {
            ECK(launch_fields(slots[j], d_fields_ + used));
            used += 5 * probs_[slots[j]].n;
        }
        ECK(cudaMemcpyAsync(h_fields_, d_fields_, sizeof(double) * used, cudaMemcpyDeviceToHost, st_));
        ECK(cudaStreamSynchronize(st_));
        int64_t off = 0;
        for (int q = i; q < j; ++q) {
            const int64_t n = probs_[slots[q]].n;
            for (int f = 0; f < 5; ++f) {
                double* dst = outs[5 * (int64_t)q + f];
                if (dst) std::memcpy(dst, h_fields_ + off + f * n, sizeof(double) * n);
            }
            off += 5 * n;
        }
        i = j;
    }
    return LBM_OK;
}

void ArenaEngine::release(int slot) {
    HostProb& p = probs_[slot];
    if (p.state == P_FREE) return;
    if (p.state == P_RUNNING) {
        --nrunning_;
        tiles_dirty_ = true;
    }
    apop_.release(p.pop_off, p.pop_bytes);
    if (dtype_ == S_F16S) acar_.release(p.car_off, p.car_bytes);
    afs_.release(p.fs_off, p.fs_bytes);
    p = HostProb();
}

// ---------------------------------------------------------------------------
// Autotuner cache: "key V" lines in $LBM_AUTOTUNE_CACHE (default
// $HOME/.cache/lbm_gb300/autotune.txt).  LBM_AUTOTUNE=0 disables lookups.
// ---------------------------------------------------------------------------

namespace {
std::mutex g_tune_mutex;

std::string cache_path() {
    const char* p = std::getenv("LBM_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char* h = std::getenv("HOME");
    std::string dir = std::string(h && *h ? h : "/tmp") + "/.cache";
    mkdir(dir.c_str(), 0755);
    dir += "/lbm_gb300";
    mkdir(dir.c_str(), 0755);
    return dir + "/autotune.txt";
}
}  // namespace

int autotune_lookup(const std::string& key) {
    const char* off = std::getenv("LBM_AUTOTUNE");
    if (off && std::string(off) == "0") return 0;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::ifstream in(cache_path());
    std::string k;
    int v = 0, found = 0;
    while (in >> k >> v)
        if (k == key) found = v;
    return found;
}

void autotune_store(const std::string& key, int V) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::ofstream out(cache_path(), std::ios::app);
    if (out) out << key << " " << V << "\n";
}

}  // namespace lbm
