// lbm_arena.cuh -- packed lattice arena for many independent periodic
// problems of uneven sizes and material parameters, advanced together by one
// persistent cooperative kernel per chunk of k steps.
//
// Every problem p owns, in three device buffers,
//   pop[0], pop[1] : its 8 population planes (ping-pong; FP32 or FP16),
//   car[0], car[1] : FP16-shifted only: the two FP32 carriers, one float2 per node,
//   fs             : force (2 FP32 planes) then residual snapshot (2 planes of
//                    (hi, lo) FP32 pairs),
// placed by a first-fit allocator (256-byte aligned).  The work of one step
// is the list of (problem, tile) pairs of the active problems; the kernel
// walks that list grid-stride, then synchronises the whole grid before the
// next step (cooperative launch).  The last step of a chunk carries the
// residual check for the problems flagged in their descriptor (a problem
// checks every `check_period` chunks of its own steps); its per-problem
// partial sums go to per-problem FP64 accumulators with atomics.  The host reads them after the chunk, retires
// converged problems, admits new ones and rebuilds the tile list between
// chunks; the chunk itself (accumulator reset, kernel, accumulator read-back)
// is replayed from a CUDA graph.
#pragma once

#include <cooperative_groups.h>

#include <map>
#include <string>
#include <vector>

#include "lbm_kernels.cuh"

namespace lbm {

struct BatchProb {
    int64_t pop_off;   // bytes into each population buffer
    int64_t car_off;   // bytes into each carrier buffer (F16S)
    int64_t fs_off;    // bytes into the force/snapshot buffer
    int nx, ny, check, dtype, parity;   // check: this chunk's last step checks
    int seg;                            // wavefront chunk: rows per wavefront item
    float q11, qs, qd, qtheta, theta, hscale, hinv;   // rates in the quarter form of collide
};

struct BatchArgs {
    const BatchProb* probs;
    const uint2* tiles;        // (problem, tile)
    const int* ntiles;         // device scalar: number of valid tiles
    const int* nwide;          // wavefront chunks: the first *nwide tiles are wavefront items
    int* counters;             // wavefront chunks: one work counter per phase, zero at launch
    char* pop0;
    char* pop1;
    char* car0;
    char* car1;
    char* fs;
    double* acc;               // kRes doubles per problem
    int nsteps;
};

constexpr int kArenaAlign = 256;

// First-fit allocator over [0, capacity) with coalescing of free ranges.
class RangeAllocator {
public:
    void reset(int64_t capacity) {
        free_.clear();
        if (capacity > 0) free_[0] = capacity;
        cap_ = capacity;
    }
    int64_t capacity() const { return cap_; }
    // returns offset or -1
    int64_t alloc(int64_t bytes) {
        bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest > 0) free_[off + bytes] = rest;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t largest_free() const {
        int64_t m = 0;
        for (auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    std::map<int64_t, int64_t> free_;
    int64_t cap_ = 0;
};

// Tile code of two-step tiles: the 62 x 22-node tiles of k_step2, two steps
// per tile visit and one grid barrier per pair of steps (chunk length even).
constexpr int kTileTwoStep = 3;

// Tile code of the wavefront chunk: problems from one strip width up advance
// four steps per visit of a wavefront item (one strip by `seg` rows);
// narrower ones take two two-step tiles per four steps (chunk length a
// multiple of 4).  The segment length is chosen when the work list is built:
// 256 rows, halved (down to 16) while the list would hold fewer than four
// waves of resident blocks, so that a few large problems still fill the GPU.
constexpr int kTileWave = 5;
constexpr int kArenaWaveSegMax = 256;

// (wavefront items address a problem with 32-bit in-plane offsets)
inline bool arena_wide(int nx, int ny) { return wave_fits(nx, ny) && (int64_t)nx * ny < (int64_t(1) << 31); }

// Relative device work per lattice update of an nx x ny problem in the
// wavefront chunk: a wide problem pays for the slot columns of its 256-column
// strips; a narrower one runs two-step tiles, at about half the wavefront's
// rate on a large lattice (GB300: 159 against 308 GLUPS), and pays for the
// slots of its tiles.
inline double arena_cost(int nx, int ny) {
    if (arena_wide(nx, ny)) return double((nx + wv_ox<4>() - 1) / wv_ox<4>()) * kWvW / nx;
    return 1.94 * (double((nx + kT2OX - 1) / kT2OX) * kT2W / nx) * (double((ny + kT2OY - 1) / kT2OY) * kT2H / ny);
}

// Solve a problem on its transpose (x and y exchanged) where that is clearly
// cheaper.  The scheme is symmetric under the exchange (velocities (c_x, c_y)
// -> (c_y, c_x) map the moments 10 <-> 01, 12 <-> 21, s -> s, d -> -d, 11 ->
// 11, 22 -> 22 onto each other; Table 1 and the rates with w_12 = w_21 follow),
// so the transposed problem's solution is the solution's transpose with u_x
// <-> u_y and sigma_xx <-> sigma_yy; only the rounding order differs.
inline bool arena_transpose(int nx, int ny) { return arena_cost(ny, nx) < 0.95 * arena_cost(nx, ny); }

// Number of tiles of an nx x ny problem for tile code V (seg: rows per
// wavefront item of the wavefront chunk).
inline int64_t arena_tiles(int nx, int ny, int V, int seg = kArenaWaveSegMax) {
    if (V == kTileWave)
        return arena_wide(nx, ny) ? (int64_t)((nx + wv_ox<4>() - 1) / wv_ox<4>()) * ((ny + seg - 1) / seg)
                                  : step2_tiles(nx, ny);
    return V == kTileTwoStep ? step2_tiles(nx, ny) : step_tiles(nx, ny, V);
}

// Launch one chunk: nsteps steps of every listed tile (all of storage type
// dtype: S_F32 or S_F16S), residual check fused into the last step.  Tile
// code V: width 32*V for V in {1, 2, 4}, kTileTwoStep or kTileWave.
// Cooperative launch: grid must not exceed arena_occupancy(dtype, V) x SM
// count.
cudaError_t launch_arena_chunk(int dtype, int V, const BatchArgs& a, int grid, cudaStream_t st);
// Resident blocks per SM of the chunk kernel.
int arena_occupancy(int dtype, int V);

}  // namespace lbm
