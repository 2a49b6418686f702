// lbm_batch.cu -- lbm_batch_solve: many independent periodic problems solved
// together in one packed arena by the persistent chunk kernel, with the tile
// width chosen by the autotuner.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_engine.cuh"

using namespace lbm;

namespace {

int bfail(int code, const std::string& m) { return set_last_error(code, m); }

std::string device_name() {
    int dev = 0;
    cudaDeviceProp p{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess)
        return "unknown";
    std::string s = p.name;
    for (auto& ch : s)
        if (ch == ' ') ch = '_';
    return s + "_sm" + std::to_string(p.multiProcessorCount);
}

// Workload signature for the autotuner cache: device, storage, check
// interval, number of problems and median side, each bucketed by powers of 2.
std::string signature(int count, const lbm_problem* probs, int dtype, int k) {
    std::vector<int> sides;
    sides.reserve(count);
    for (int i = 0; i < count; ++i) sides.push_back(std::max(probs[i].nx, probs[i].ny));
    std::nth_element(sides.begin(), sides.begin() + count / 2, sides.end());
    const int med = sides[count / 2];
    auto lg = [](double v) { return (int)std::floor(std::log2(std::max(v, 1.0))); };
    return device_name() + "|d" + std::to_string(dtype) + "|k" + std::to_string(k) + "|n" +
           std::to_string(lg(count)) + "|s" + std::to_string(lg(med));
}

}  // namespace

extern "C" int lbm_batch_solve(int count, const lbm_problem* probs, int dtype, double tol,
                               int check_every, int64_t max_iters, lbm_result* results,
                               lbm_batch_report* report) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (count < 1 || !probs || !results)
        return bfail(LBM_ERR_ARG, "lbm_batch_solve: need count >= 1 and non-null arrays");
    if (dtype != LBM_F32 && dtype != LBM_F16S)
        return bfail(LBM_ERR_ARG, "lbm_batch_solve: dtype must be LBM_F32 or LBM_F16S");
    if (!(tol >= 0.0) || check_every < 2 || max_iters < 1)
        return bfail(LBM_ERR_ARG, "lbm_batch_solve: need tol >= 0, check_every >= 2, max_iters >= 1");
    int64_t nodes = 0;
    for (int i = 0; i < count; ++i) {
        const lbm_problem& p = probs[i];
        if (p.nx < 1 || p.ny < 1 || !p.gx || !p.gy || !(p.mu > 0.0) || !(p.lambda + p.mu > 0.0))
            return bfail(LBM_ERR_ARG, "lbm_batch_solve: problem " + std::to_string(i) + " is invalid");
        nodes += (int64_t)p.nx * p.ny;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return bfail(LBM_ERR_CUDA, "lbm_batch_solve: stream creation failed");
    std::string err;
    int rc;
    int chosen_V = 0, grid = 0;
    int64_t chunks = 0, lups = 0;
    double dev_ms = 0.0;
    {
        ArenaEngine eng;
        rc = eng.init(dtype, nodes, count, check_every, st, &err);
        if (rc) {
            cudaStreamDestroy(st);
            return bfail(rc, "lbm_batch_solve: " + err);
        }
        std::vector<int> slot(count);
        for (int i = 0; i < count && rc == LBM_OK; ++i) {
            const lbm_problem& p = probs[i];
            int s = eng.admit(p.nx, p.ny, p.lambda, p.mu, p.gx, p.gy, tol, max_iters, &err);
            if (s == -1) rc = LBM_ERR_OOM, err = "arena full";
            else if (s < 0) rc = s;
            slot[i] = s;
        }
        // Autotuner: the first chunks run with tile widths 32, 64 and 128
        // and, for an even chunk length, with two-step tiles; the fastest per
        // active node and chunk is kept and cached.
        const std::string key = signature(count, probs, dtype, check_every);
        const bool even = check_every % 2 == 0, four = check_every % 4 == 0;
        int V = rc == LBM_OK ? autotune_lookup(key) : 0;
        if ((V == kTileTwoStep && !even) || (V == kTileWave && !four)) V = 0;
        if (const char* force_v = std::getenv("LBM_BATCH_TILE_V")) {  // fixed shape, no tuning
            const int fv = std::atoi(force_v);
            if (fv == 1 || fv == 2 || fv == 4 || (fv == kTileTwoStep && even) || (fv == kTileWave && four))
                V = fv;
        }
        // candidates, the likeliest first (the wavefront chunk when the chunk
        // length allows it)
        int cand[5], ncand = 0;
        if (four) cand[ncand++] = kTileWave;
        if (even) cand[ncand++] = kTileTwoStep;
        cand[ncand++] = 4;
        cand[ncand++] = 2;
        cand[ncand++] = 1;
        double best = 1e300;
        int tuning = V == 0 ? 0 : ncand;
        while (rc == LBM_OK && eng.running() > 0) {
            const int v = tuning < ncand ? cand[tuning] : V;
            const int64_t active_nodes = eng.running_nodes();
            float ms = 0.0f;
            rc = eng.run_chunk(v, &ms, &err);
            if (rc) break;
            ++chunks;
            dev_ms += ms;
            if (tuning < ncand) {
                const double per = ms / (double)std::max<int64_t>(active_nodes, 1);
                if (per < best) {
                    best = per;
                    V = v;
                }
                if (++tuning == ncand) autotune_store(key, V);
            }
        }
        chosen_V = V;
        grid = V ? eng.grid_blocks(V) : 0;
        if (rc == LBM_OK) {
            // problems whose caller wants fields, recovered together
            std::vector<int> want;
            std::vector<double*> outs;
            for (int i = 0; i < count; ++i) {
                const HostProb& hp = eng.prob(slot[i]);
                lbm_result& r = results[i];
                r.status = hp.status;
                r.iters = hp.steps;
                r.residual = hp.residual;
                r.transposed = hp.tr ? 1 : 0;
                lups += hp.lups;
                double* o[5] = {r.ux, r.uy, r.sxx, r.syy, r.sxy};
                if (!(o[0] || o[1] || o[2] || o[3] || o[4])) continue;
                want.push_back(slot[i]);
                outs.insert(outs.end(), o, o + 5);
            }
            rc = eng.recover_many((int)want.size(), want.data(), outs.data(), &err);
        }
    }
    cudaStreamDestroy(st);
    if (report) {
        report->tile_v = chosen_V;
        report->blocks = grid;
        report->chunks = chunks;
        report->lattice_updates = lups;
        report->device_ms = dev_ms;
        report->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    }
    if (rc) return bfail(rc, "lbm_batch_solve: " + err);
    return LBM_OK;
}
