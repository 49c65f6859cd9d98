// Internal definition of a grid (one room) shared by the C ABI (capi.cpp) and the batch engine (batch.cpp).
#pragma once

#include <cuda_runtime_api.h>

#include <string>
#include <vector>

#include "vf_internal.h"

struct vf_grid {
    vf_grid_desc d{};
    bool fp64 = false;
    size_t N = 0, esz = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    vf_allocator alloc{};
    bool have_alloc = false;
    std::vector<void*> allocs;
    size_t bytes = 0;
    int alloc_count = 0;
    int fail_alloc_at = 0;       // fault injection: the n-th allocation of this grid fails (0 = off)

    void* q = nullptr;           // state (u, v, w, c) per cell as a 4-vector
    void* acc = nullptr;         // RK4 stage states (q2, q3, q4 and q*; see enqueue_step)
    void* qa = nullptr;
    void* qb = nullptr;
    void* p = nullptr;
    void* f = nullptr;           // right-hand side of Eq. 9: D u* / dt, plus the correction next to solids
    void* spec = nullptr;
    int* near_list = nullptr;    // cells with a solid axis neighbour, ascending (capacity N)
    void* near_r = nullptr;      // D u* / dt at those cells (capacity N)
    int n_near = 0;
    bool plane_layout = false;
    // register path of the Poisson solve (PoissonArgs::reg and its shape), fixed at creation
    int reg = 0, reg_rx = 0, reg_ry = 0, reg_rz = 0, reg_gx = 0, reg_gy = 0, reg_gz = 0, reg_sp = 0, reg_spx = 0, reg_sb = 0;
    int reg_tile = 0, reg_sy = 0, reg_tb = 0, reg_st = 0;
    void* staging = nullptr;     // N * 8 bytes
    uint8_t* mask = nullptr;
    uint8_t* smask = nullptr;    // stencil mask of the stage kernels (rebuilt whenever beta or S change)
    void* sval = nullptr;        // smooth forcing region values (Eq. 5 or caller's), N values of the precision
    bool smooth_s = false;       // the stage kernels take S from sval (else S = 1 on the S bit)
    void* target = nullptr;      // per-cell forcing targets (u, v, w, c) as a 4-vector array, allocated on first use
    bool has_target = false;     // the stage kernels take the targets from `target` (the constants are then 0)
    double* force_acc = nullptr; // vf_region_force accumulators [3]
    void* twx = nullptr;
    void* twy = nullptr;
    void* twz = nullptr;
    void* twr = nullptr;
    void* lamx = nullptr;
    void* lamy = nullptr;
    void* lamz = nullptr;
    int* krev_y = nullptr;       // digit-reversal tables of the in-place y and z transforms
    int* krev_z = nullptr;

    double* red_partial = nullptr;
    double* div_partial = nullptr;       // the filter's per-warp records (divergence, mask loss, room change)
    double* budget_partial = nullptr;    // scalar budget: CTA partials of stages 3 and 4, ticket, the step's terms
    unsigned int* budget_done = nullptr;
    double* budget_out = nullptr;
    int* budget_list = nullptr;          // cells with the budget bit, ascending (capacity N)
    int n_budget = 0;
    unsigned long long* hist_accum = nullptr;
    unsigned int* red_done = nullptr;
    vf_reduce* red_out = nullptr;
    vf_reduce* history = nullptr;
    long long* dev_counters = nullptr;   // [0] history count, [1] step counter
    int* nonfinite = nullptr;
    vf::DtCtl* dtctl = nullptr;          // time-step control (read by the kernels only with a dynamic dt)
    vf::ParticleArgs particles{};        // Lagrangian particles (n = 0: none); arrays in one buffer
    void* particle_buf = nullptr;
    size_t particle_bytes = 0;
    bool dynamic = false;                // courant_max > 0
    bool sigma_stale = true;             // the Courant rate of the current state must be recomputed
    unsigned long long* solid_count = nullptr;
    int nred = 0;
    int ndiv = 0;

    int zc[vf::kZcKinds] = {4, 32, 8, 16};  // z-chunks (vf_tiles): stage, divergence, projection, filter

    int fft_sched[3] = {0, 0, 0};          // radix schedule index per axis (vf_tiles fft_x, fft_y, fft_z)
    vf::FftAxis ax{}, ay{}, az{};
    int rows_per_block = 1, cols_per_block = 16;

    cudaGraphExec_t gexec[4]{nullptr, nullptr, nullptr, nullptr};   // step graphs (see capture_graphs)
    cudaStream_t side_stream = nullptr;  // the previous step's reduction alongside stages 1-2
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool graph_ok = false;
    bool use_graph = true;

    int status = VF_OK;
    std::string err;
    bool mask_set = false;
    bool has_solid = false;
    double uset[3]{0, 0, 0};
    double cset = 0;
    int64_t step = 0;
    double t0 = 0;
};


namespace vf_engine {

// Dynamic time step: recompute the Courant rate of the current state on stream st if a field changed since the
// last step (no-op otherwise).
cudaError_t refresh_sigma(vf_grid* g, cudaStream_t st);

// Enqueue one step of grid g on stream st (with the FP64 reductions if with_reduce); the launches a single-room
// vf_step replays.  Returns the first CUDA error.
cudaError_t enqueue_step(vf_grid* g, cudaStream_t st, bool with_reduce);

// Device bytes vf_create_grid allocates for a description (each buffer rounded up to 256 bytes).
size_t grid_bytes(const vf_grid_desc& d);

}  // namespace vf_engine
