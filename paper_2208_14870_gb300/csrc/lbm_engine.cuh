// lbm_engine.cuh -- host side of the packed lattice arena: admission of
// problems into arena slots, chunk replay (CUDA graph around the persistent
// cooperative kernel), per-problem residual bookkeeping, retirement and
// solution recovery.  Shared by lbm_batch_solve and the serving loop.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm_arena.cuh"

namespace lbm {

enum ProbState { P_FREE = 0, P_RUNNING = 1, P_DONE = 2 };

struct HostProb {
    int state = P_FREE;
    int nx = 0, ny = 0;            // the arena lattice (the caller's, or its transpose)
    bool tr = false;               // solved transposed (arena_transpose)
    int64_t n = 0;
    double lambda = 0.0, mu = 0.0;
    int64_t pop_off = -1, car_off = -1, fs_off = -1;
    int64_t pop_bytes = 0, car_bytes = 0, fs_bytes = 0;
    int parity = 0;
    int hexp = 0;
    float q11 = 0, qs = 0, qd = 0, qtheta = 0, theta = 0;   // rates in the quarter form of collide
    int64_t steps = 0;
    int64_t max_iters = 0;
    double tol = 0.0;
    bool snap_valid = false;
    bool check_now = false;    // the coming chunk checks this problem
    int period = 1;            // residual window = period chunks (adapt_period)
    int64_t last_check = 0;    // steps at the previous check
    double r_prev = 0.0;       // residual of the previous check
    int status = 0;            // lbm status when done
    double residual = 0.0;
    int64_t lups = 0;          // nodes x steps
};

class ArenaEngine {
public:
    ~ArenaEngine();
    // dtype: S_F32 or S_F16S.  Capacities in nodes (population / carrier /
    // force+snapshot bytes follow from the storage type).
    int init(int dtype, int64_t node_capacity, int max_probs, int check_every, cudaStream_t st,
             std::string* err);
    int dtype() const { return dtype_; }
    int check_every() const { return k_; }
    // Bytes of device memory a problem of n nodes needs in this arena.
    int64_t bytes_for(int64_t n) const;
    // Admit a problem; returns slot >= 0, -1 if it does not fit now, or a
    // negative lbm status (< -1) on error.  gx, gy: host FP64, nx*ny each.
    int admit(int nx, int ny, double lambda, double mu, const double* gx, const double* gy,
              double tol, int64_t max_iters, std::string* err);
    // One chunk of check_every steps for every running problem; afterwards
    // finished problems are in state P_DONE (not yet released).
    int run_chunk(int V, float* device_ms, std::string* err);
    // Solution fields of a finished (or running) problem into host arrays
    // (nullable), FP64, lattice units.
    int recover(int slot, double* ux, double* uy, double* sxx, double* syy, double* sxy,
                std::string* err);
    // The same for count problems at once; outs holds 5 nullable host arrays
    // (ux, uy, sxx, syy, sxy) per problem.  Few copies and synchronisations.
    int recover_many(int count, const int* slots, double* const* outs, std::string* err);
    void release(int slot);
    const HostProb& prob(int slot) const { return probs_[slot]; }
    int running() const { return nrunning_; }
    int64_t running_tiles(int V, int seg = kArenaWaveSegMax) const;
    int64_t running_nodes() const;
    // Arena bytes held by admitted problems (running or finished, not released).
    int64_t resident_bytes() const;
    int max_probs() const { return (int)probs_.size(); }
    int grid_blocks(int V) const;
    int64_t free_nodes_hint() const;
    int64_t device_bytes() const { return dev_bytes_; }
    cudaStream_t stream() const { return st_; }

private:
    int upload_tiles(int V, std::string* err);
    BatchArgs chunk_args() const;
    cudaError_t launch_fields(int slot, double* dst);
    int ensure_fields_buffer(int64_t len, std::string* err);
    int ensure_graph(int V, std::string* err);

    int dtype_ = S_F32;
    int k_ = 100;
    cudaStream_t st_ = nullptr;
    int sms_ = 1;
    char* pop_[2] = {nullptr, nullptr};
    char* car_[2] = {nullptr, nullptr};
    char* fs_ = nullptr;
    RangeAllocator apop_, acar_, afs_;
    std::vector<HostProb> probs_;
    BatchProb* d_probs_ = nullptr;
    double* d_acc_ = nullptr;
    double* h_acc_ = nullptr;         // pinned
    uint2* d_tiles_ = nullptr;
    int64_t tiles_cap_ = 0;
    int* d_ntiles_ = nullptr;
    int* d_nwide_ = nullptr;          // wavefront chunks: wavefront items at the list's head
    int* d_counters_ = nullptr;       // wavefront chunks: a work counter per phase (2 per pass)
    uint2* h_tiles_ = nullptr;        // pinned
    int64_t h_tiles_cap_ = 0;
    int tiles_V_ = 0;                 // V the device tile list was built for
    int wave_seg_ = kArenaWaveSegMax; // rows per wavefront item of the current list
    bool tiles_dirty_ = true;
    bool desc_dirty_ = true;
    float* h_force_ = nullptr;        // pinned FP32 staging
    int64_t h_force_cap_ = 0;
    double* d_fields_ = nullptr;      // FP64 staging for recovery
    int64_t d_fields_cap_ = 0;
    double* h_fields_ = nullptr;      // pinned block for recover_many
    cudaGraphExec_t graph_[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool graph_failed_[6] = {false, false, false, false, false, false};
    cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
    int nrunning_ = 0;
    int64_t dev_bytes_ = 0;
};

// Message for lbm_last_error() on this host thread; returns code.
int set_last_error(int code, const std::string& msg);

// Autotuner cache: tile width chosen for a workload signature.
int autotune_lookup(const std::string& key);
void autotune_store(const std::string& key, int V);

}  // namespace lbm
