// Internal interfaces between the C ABI / step engine (capi.cpp, host C++) and the CUDA kernels (*.cu).
// Only plain structs and host launchers appear here, so capi.cpp compiles with a host compiler.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime_api.h>

#include "../../include/ventflow.h"

namespace vf {

constexpr int kHistBins = 64;
constexpr int kMaxRadixStages = 16;

// Mask byte of a cell: bit 0 beta (fluid), bit 1 S (forcing region), bit 2 room region, bit 3 "a neighbour
// along some axis is solid" (derived from beta by vf_set_mask; the Eq. 9 correction is zero without it).
constexpr uint8_t kBitBeta = 1u;
constexpr uint8_t kBitS = 2u;
constexpr uint8_t kBitRoom = 4u;
constexpr uint8_t kBitNearSolid = 8u;
constexpr uint8_t kBitForce = 16u;   // cells whose immersed-boundary force vf_region_force sums
// cells that enter the scalar budget of the stages: fluid forcing cells, and fluid room cells with a fluid axis
// neighbour outside the room (a face of the room's boundary); derived from beta, S and the room bits
constexpr uint8_t kBitBudget = 32u;

// Stencil mask of the stage kernels: one byte per cell with its own beta and S bits and the beta of its six axis
// neighbours, so a cell's stencil reads one byte instead of five.
constexpr uint8_t kSmSelf = 1u, kSmS = 2u, kSmXm = 4u, kSmXp = 8u, kSmYm = 16u, kSmYp = 32u, kSmZm = 64u,
                  kSmZp = 128u;

// Constants of the flow kernels, in the compute precision T.
// Kernel families with their own z-chunk (planes one CTA marches along z); the allowed range of a chunk.
enum ZcKind { kZcStage = 0, kZcDiv = 1, kZcProject = 2, kZcFilter = 3, kZcKinds = 4 };
constexpr int kZChunkMin = 4;
constexpr int kZChunkMax = 64;

// Device-resident control of a dynamic time step (Sec. 2.4: the user sets the maximum Courant number and AdjustDt
// adapts dt).  The adjust kernel at the start of every step reads sigma_bits (max over cells of sum_j |u_j| / h_j
// of the state the step starts from), chooses dt = min(dt_max, courant_max / sigma), writes the dt-dependent
// constants below with the same formulas the host uses for a fixed dt, advances the time and clears sigma_bits
// for the kernel that writes the step's final state.  All in double; kernels convert to their precision.
struct DtCtl {
    double dt;                    // time step of the current step
    double t_end;                 // simulated time at the end of the current step
    double dt2, dt3, dt6;         // dt / 2, dt / 3, dt / 6
    double inv_tau;               // 1 / tau_f (tau_f <= 0: 1 / dt)
    double i2h_div[3];            // 1 / (2 h_j dt)
    double i2h_dt[3];             // dt / (2 h_j)
    unsigned long long sigma_bits;   // double bits of the Courant rate (non-negative: bit order = value order)
    double courant_max, dt_max, tau_f;
    double h[3];
};

template <typename T>
struct FlowConsts {
    int nx, ny, nz;
    int zc[kZcKinds]; // z-chunk per kernel family (the filter's also sets the reduction's CTAs)
    T i2h[3];     // 1 / (2 h_j)
    T i2h_div[3]; // 1 / (2 h_j dt): the divergence is stored divided by dt
    T i2h_dt[3];  // dt / (2 h_j): the pressure is stored as p / rho, the projection subtracts dt G p
    T q4h[3];     // 1 / (4 h_j): the 1/2 of the skew form times the 1/(2h) of the central difference
    T ih[3];      // 1 / h_j
    T ih2[3];     // 1 / h_j^2
    T nu, alpha, inv_tau;
    T dt6, dt3, dt2, dt;  // dt/6, dt/3, dt/2, dt
    T third;              // 1/3
    T bf[3];      // body force
    T uset[3];    // forcing target velocity
    T cset;       // forcing target scalar
    T filt;       // pi^-6
    const DtCtl* dyn;   // dynamic time step: dt-dependent constants come from here (nullptr: the fields above)
};

// Scalar budget of a step's four stage states (Eqs. 3-4 in flux form, the room inventory of Sec. 3.3), computed
// by extra CTAs of the stage 3 and stage 4 launches on steps that write a reduction record: stage 3's read q_n and
// q2, stage 4's q3 and q4, none of which that launch writes.  The CTA partials of both launches are added in CTA
// order by the last budget CTA of stage 4 (atomic ticket).
struct BudgetArgs {
    int n = -1;               // cells in the list; < 0: no budget CTAs in this launch
    int ctas = 0;             // budget CTAs of this launch (at least 1 when n >= 0)
    int ctas_prev = 0;        // budget CTAs of the stage 3 launch (stage 4 adds their partials too)
    int slot = 0;             // 0: stage 3 launch, 1: stage 4 launch
    int cap = 0;              // CTA partials per slot
    const int* list = nullptr;        // cells with the budget bit, ascending
    const void* qa = nullptr;         // the two stage states of this launch and their RK4 weights
    const void* qb = nullptr;
    double wa = 0.0, wb = 0.0;
    double* partial = nullptr;        // [2][cap][kBudgetTerms]
    unsigned int* done = nullptr;     // ticket of stage 4's budget CTAs, zero between launches
    double* out = nullptr;            // [kBudgetTerms] of the step, scaled by dt and dV
    double dV = 0.0, dt = 0.0, inv_tau = 0.0, alpha = 0.0, cset = 0.0, ih[3] = {0.0, 0.0, 0.0};   // in double;
                                      // a dynamic step takes dt and 1 / tau_f from DtCtl
};

// Pointers of one RK4 stage.  Every state array holds one 4-vector (u, v, w, c) of T per cell (16 bytes for
// float, 32 for double): q_s (stencil input), q_n, the stage states q2, q3 (read by stage 4) and the output.
template <typename T>
struct StageArgs {
    const void* qs;
    const void* qn;
    const void* q2;
    const void* q3;
    void* out;
    const uint8_t* mask;
    const uint8_t* smask;   // stencil mask (kSm* bits)
    const T* sval;      // smooth forcing region S in [0, 1] at the cells whose S bit is set (nullptr: S = 1 there)
    const void* target; // per-cell forcing targets (u, v, w, c)_set as a 4-vector array (nullptr: the constants;
                        // when given, the constants are 0 and S beta target / tau_f is added at the S cells)
    BudgetArgs bud;     // stages 3 and 4 of a recorded step: the scalar budget CTAs
};

// One smooth source window of Eq. 5 on a grid: centre c_j, half widths W_j / 2, sharpness B_j, cell size h_j and
// box length L_j per axis (x, y, z).
struct TanhWindow {
    double c[3], hw[3], B[3], h[3], L[3];
};

// Division by a run-time invariant d by multiply and shift (Granlund-Montgomery), exact for n < 2^31.
struct FastDiv {
    uint32_t d, m, s;
};

inline FastDiv make_fast_div(uint32_t d)
{
    FastDiv f{d, 0u, 0u};
    if (d <= 1) return f;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;                       // l = ceil(log2 d)
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s = l;
    return f;
}

// One radix pass of a Stockham FFT of length n: R-point butterflies over n / R groups; Ns = product of the
// radices already applied; twiddle exponent stride n / (Ns R).
// The same stage read as an in-place decimation-in-frequency pass: sub-length L = n / Ns, R groups of
// m = L / R = tstride elements, twiddle W_L^(j k) = W_n^(j k Ns).
struct FftStage {
    int R, Ns, nb, tstride;
    FastDiv ns_div;   // j -> j / Ns
    FastDiv nb_div;   // item -> item / nb (row-batched passes)
    FastDiv m_div;    // item -> item / tstride (in-place passes)
};

// One FFT axis: length and radix schedule (product of the radices == n).  The power-of-two part takes as few
// passes as possible: radix-16 passes where they need fewer passes than radix 8 (e.g. 128 = 16 x 8), otherwise
// radix-8 passes with a remainder of 2 as 4 x 4 or a 4; then the factors 3 and 5.
struct FftAxis {
    int n;
    int nstages;
    FftStage st[kMaxRadixStages];
};

inline FftAxis make_fft_axis(int n)
{
    FftAxis a{};
    a.n = n;
    int rad[kMaxRadixStages], k = 0;
    int m = n, twos = 0;
    while (m % 2 == 0) { m /= 2; ++twos; }
    const int p16 = (twos + 3) / 4, p8 = (twos + 2) / 3;
    if (twos >= 4 && p16 < p8) {
        // p16 passes: radix 16 while at least 4 factors of two remain for it, the rest as 8, 4 or 2
        int left = twos;
        for (int i = 0; i < p16 && k < kMaxRadixStages; ++i) {
            const int passes_left = p16 - i;
            const int e = (left + passes_left - 1) / passes_left >= 4 ? 4 : (left + passes_left - 1) / passes_left;
            rad[k++] = 1 << e;
            left -= e;
        }
    } else {
        int eights = twos / 3;
        const int rem = twos % 3;
        if (rem == 1 && eights > 0) { --eights; rad[k++] = 4; rad[k++] = 4; }
        else if (rem == 1) rad[k++] = 2;
        else if (rem == 2) rad[k++] = 4;
        for (int i = 0; i < eights && k < kMaxRadixStages; ++i) rad[k++] = 8;
    }
    while (m % 3 == 0 && k < kMaxRadixStages) { m /= 3; rad[k++] = 3; }
    while (m % 5 == 0 && k < kMaxRadixStages) { m /= 5; rad[k++] = 5; }
    a.nstages = k;
    int Ns = 1;
    for (int s = 0; s < k; ++s) {
        FftStage& S = a.st[s];
        S.R = rad[s];
        S.Ns = Ns;
        S.nb = n / S.R;
        S.tstride = n / (Ns * S.R);
        S.ns_div = make_fast_div((uint32_t)Ns);
        S.nb_div = make_fast_div((uint32_t)S.nb);
        S.m_div = make_fast_div((uint32_t)S.tstride);
        Ns *= S.R;
    }
    return a;
}

// Everything one Poisson iteration needs.  Two spectrum layouts, (nx/2) x ny x nz complex values in both:
//   tile  : [z][y][kx], kx fastest; the y and z passes work on tiles of cols_per_block consecutive kx columns;
//   plane : [kx][z][y], y fastest; one CTA per kx transforms its whole (y, z) plane in shared memory (y FFT,
//           z FFT, eigenvalue division, inverse z and y FFTs), used when a plane fits in one CTA.
// Column kx = 0 packs the real spectra at kx = 0 (real part) and kx = nx/2 (imaginary part).
template <typename T>
struct PoissonArgs {
    int nx, ny, nz, M;        // M = nx / 2
    T* f;                     // right-hand side read by the x forward pass (r, plus the Eq. 9 correction)
    T* p;                     // in: p^k (for the correction), out: p^{k+1}
    const uint8_t* smask;     // packed stencil mask: the betas of each cell's six axis neighbours (kSm* bits)
    const int* near_list;     // ascending cells with a solid axis neighbour (where the correction is nonzero)
    T* near_r;                // r at those cells, saved by the first correction of a step
    int n_near;
    int plane_layout;
    void* spec;               // complex T [M * ny * nz]
    const void* twx;          // complex T [M]:  exp(-2 pi i m / M)
    const void* twy;          // complex T [ny]
    const void* twz;          // complex T [nz]
    const void* twr;          // complex T [M + 1]: exp(-2 pi i k / nx), real-FFT packing twiddles
    const T* lamx;            // [M]  sin^2(2 pi kx / nx) / hx^2 (kx = 0 and nx/2 share column 0, both 0)
    const T* lamy;            // [ny]
    const T* lamz;            // [nz]
    const int* krev_y;        // [ny] spectral index held at each position after the in-place forward y FFT
    const int* krev_z;        // [nz]
    T i2h2[3];                // (1 / (2 h_j))^2
    T invN;                   // 1 / (nx ny nz)
    FftAxis ax, ay, az;
    FastDiv ny_div;           // i -> i / ny (plane passes)
    FastDiv nx_div;           // i -> i / nx (cell index -> row, correction kernel)
    int rows_per_block;       // rows of the x passes per CTA
    int cols_per_block;       // kx columns of the y / z tile passes per CTA
    // register path (every axis length R G: 16 G with G in 1, 2, 4, 8, 16, and in FP32 the 2-3-5 lengths 36 .. 96):
    // the transforms are held in registers, G threads per sequence with R values each; whole-plane kernel when the
    // (y, z) plane of one kx fits in shared memory, else tile mode (16 G lengths only)
    int reg;
    int rx, ry, rz;           // values per thread of the x (M points), y and z transforms
    int gx, gy, gz;           // threads per transform: M = rx gx, ny = ry gy, nz = rz gz
    int reg_sp;               // complex stride between the z rows of the shared plane
    int reg_spx;              // complex stride between the rows of the x passes
    int reg_sb;               // unused (0)
    int reg_tile;             // 1: y pass, z tile pass, y pass instead of the whole-plane kernel
    int reg_sy;               // complex stride between the rows of the y passes (tile mode)
    int reg_tb;               // y slots per z tile (tile mode)
    int reg_st;               // complex stride between the z rows of a z tile (tile mode)
};


// Spectral index at each position after the in-place (decimation-in-frequency) forward FFT of an axis: the
// position p = d_0 n/R_0 + d_1 n/(R_0 R_1) + ... holds frequency k = d_0 + R_0 (d_1 + R_1 (d_2 + ...)).
inline void digit_reversal(const FftAxis& ax, int* out)
{
    for (int p = 0; p < ax.n; ++p) {
        int rem = p, L = ax.n, k = 0, mult = 1;
        for (int s = 0; s < ax.nstages; ++s) {
            const int m = L / ax.st[s].R;
            const int d = rem / m;
            rem -= d * m;
            k += d * mult;
            mult *= ax.st[s].R;
            L = m;
        }
        out[p] = k;
    }
}

// Block size of the plane kernel (one CTA per kx plane, the plane in shared memory, at most 200 KB).
constexpr int kPlaneThreads = 512;

// Reduction scratch: per-CTA partial sums and histogram counts, and the output records.
struct ReduceArgsDev {
    double* partial;          // [kRedSlots * nblocks], quantity-major
    double* div_partial;      // the filter's records, kDivRecord per warp
    int div_count;            // records k_reduce_state folds (set by its launcher)
    unsigned long long* hist_accum;   // [kHistBins + 2], zero between launches
    unsigned int* done;       // CTAs finished in the current launch, zero between launches
    vf_reduce* out;           // single record (vf_reductions)
    vf_reduce* history;       // ring buffer
    long long* hist_count;    // records written so far
    long long* step_counter;  // device step counter
    int* nonfinite;           // set to 1 when a NaN / Inf is seen
    long long history_capacity;
    double dV;
    double dt;
    double t0;                // simulated time at step 0
    const DtCtl* dyn;         // dynamic time step: time and dt of the record from here (nullptr: t0 + step dt)
    // scalar budget of the step (nullptr: the record's budget fields are 0): the stage terms k_budget left in
    // budget[0..kBudgetTerms), and whether the filter's records carry its mask loss and room change
    const double* budget;
    int filter_budget;
};
// ke, div2, c_total, c_room, c2_room, v_room, div_max, u_max, filter mask loss, filter room change
constexpr int kRedSlots = 10;
// The filter's record per warp: sum d^2, max |d| (divergence of its input), the scalar it puts into solid cells
// (removed by the re-mask) and its change of the room cells' scalar.
constexpr int kDivRecord = 4;
// Scalar budget of the RK4 stages: forcing, forcing in the room, outflow from the room.
constexpr int kBudgetTerms = 3;

// Called after each launch of a step when a step is profiled (pass = VF phase id, see vf_phase_name).
struct LaunchHook {
    void (*fn)(void* ctx, int phase);
    void* ctx;
    void operator()(int phase) const { if (fn) fn(ctx, phase); }
};

// Stencil mask from the cell mask (beta and S bits of each cell and beta of its axis neighbours).
cudaError_t build_stencil_mask(const uint8_t* mask, uint8_t* smask, int nx, int ny, int nz, cudaStream_t st);

// Immersed-boundary force on the cells with the kBitForce bit (flow_kernels.cu): sum over them of the unmasked
// momentum right-hand side (-convection + nu diffusion + forcing + body force - grad p) times dV, into acc[3].
template <typename T>
cudaError_t region_force(const void* q, const T* p, const uint8_t* mask, const T* sval, const void* target,
                         const FlowConsts<T>& k, double dV, double* acc, cudaStream_t st);

// Lagrangian particles of a grid (Sec. 2.3; particles.cu): structure-of-arrays double state on the device.
struct ParticleArgs {
    long long n;
    double* pos[3];             // x, y, z [m], in [0, L_j)
    double* vel[3];             // u_p [m/s]
    const double* size;         // d [m] in tau_p = rho_p d^2 / (18 rho_f nu)
    int* state;                 // 0 airborne, 1 deposited
    int nx, ny, nz;
    double h[3], ih[3], L[3];
    double nu, rho_p, rho_f, g[3];
    double dt;                  // fixed time step (dyn == nullptr)
    const DtCtl* dyn;           // dynamic time step: dt of the current step from here
};

// Advance every airborne particle by one step in the velocity of the state q (4-vector array of precision T).
template <typename T>
cudaError_t advance_particles(const ParticleArgs& P, const void* q, const uint8_t* mask, cudaStream_t st);

// The adjust kernel of a dynamic time step (one thread; see DtCtl).
cudaError_t adjust_dt(DtCtl* c, cudaStream_t st);

// Register path of the Poisson solve: eligibility and launch (fft_reg.cu).
template <typename T>
struct RegFft {
    static bool eligible(int nx, int ny, int nz);              // axis lengths and shared-memory fit
    static void configure(PoissonArgs<T>& a);                   // sets reg, g*, strides (a.reg = 0 if ineligible)
    static cudaError_t prepare(const PoissonArgs<T>& a);        // shared-memory limits; call outside capture
    static cudaError_t iteration(const PoissonArgs<T>& a, cudaStream_t st, const LaunchHook* hook);
};

template <typename T>
struct Kernels {
    // s = 3, 4 with a.bud.n >= 0: plus a.bud.ctas budget CTAs (a first z slice of the grid)
    static cudaError_t stage(int s, const StageArgs<T>& a, const FlowConsts<T>& k, cudaStream_t st);
    static int budget_cta_capacity(const FlowConsts<T>& k);   // CTAs one z slice of the stage grid has
    static cudaError_t divergence(const void* qstar, T* r, const FlowConsts<T>& k, cudaStream_t st);
    // u = beta (u* - dt G p), c* passes through; ticks the device step counter
    // sigma != nullptr: also the Courant rate of the written velocity into *sigma (atomic max of double bits)
    static cudaError_t project(const void* qstar, const T* p, void* out, const uint8_t* mask, long long* step_counter,
                               const FlowConsts<T>& k, cudaStream_t st, unsigned long long* sigma = nullptr);
    // r != nullptr: also the divergence records of the projected velocity (r->div_partial) for reduce_state
    static cudaError_t filter(const void* in, void* out, const uint8_t* mask, const FlowConsts<T>& k,
                              const ReduceArgsDev* r, cudaStream_t st, unsigned long long* sigma = nullptr);
    static int filter_warps(const FlowConsts<T>& k);   // divergence records one filter launch writes
    // reductions of the filtered state q with the divergence records of the filter launched before it with the same
    // k; max_blocks: the partial slots of r (reduce_blocks)
    static cudaError_t reduce_state(const void* q, const uint8_t* mask, const FlowConsts<T>& k, ReduceArgsDev r,
                                    int to_history, int max_blocks, cudaStream_t st);
    // Eq. 5 window into the smooth forcing values and the mask's S bits (S > 0)
    static cudaError_t tanh_source(T* sval, uint8_t* mask, const TanhWindow& w, int nx, int ny, int nz,
                                   cudaStream_t st);
    // the mask's S bits from smooth forcing values (S > 0)
    static cudaError_t source_bits(uint8_t* mask, const T* sval, size_t n, cudaStream_t st);
    // Courant rate of a state into *sigma (atomic max; the caller clears it)
    static cudaError_t courant_rate(const void* q, const FlowConsts<T>& k, size_t n, unsigned long long* sigma,
                                    cudaStream_t st);
    static cudaError_t reduce(const void* q, const uint8_t* mask, const FlowConsts<T>& k, const ReduceArgsDev& r,
                              int to_history, cudaStream_t st);
    static int reduce_blocks(const FlowConsts<T>& k);
    static cudaError_t poisson_prepare(const PoissonArgs<T>& a);   // shared-memory limits; call outside capture
    // one iteration of Eq. 9; `first` marks the first iteration of a step (saves r at the near-solid cells)
    static cudaError_t poisson_iteration(const PoissonArgs<T>& a, int first, cudaStream_t st,
                                         const LaunchHook* hook = nullptr);
    static bool plane_fits(int ny, int nz);
    // component comp (0..3) of a 4-vector state array, or a scalar array when comp < 0
    static cudaError_t convert_in(const void* src, int src_fp64, void* dst, int comp, size_t n, double scale,
                                  const uint8_t* mask, cudaStream_t st);
    static cudaError_t convert_out(const void* src, int comp, void* dst, int dst_fp64, size_t n, double scale,
                                   cudaStream_t st);
    static cudaError_t apply_mask(void* q4, const uint8_t* mask, size_t n, cudaStream_t st);
    static size_t fft_smem_x(const PoissonArgs<T>& a);
    static size_t fft_smem_yz(const PoissonArgs<T>& a, int n, int buffers);
    static size_t fft_smem_plane(const PoissonArgs<T>& a);
};

// Mask helpers (precision independent).
cudaError_t mask_merge(uint8_t* mask, const uint8_t* src, uint8_t bit, size_t n, cudaStream_t st);
cudaError_t mask_fill(uint8_t* mask, uint8_t value, size_t n, cudaStream_t st);
cudaError_t mask_count_solid(const uint8_t* mask, size_t n, unsigned long long* d_count, cudaStream_t st);
cudaError_t mask_mark_near_solid(uint8_t* mask, int nx, int ny, int nz, cudaStream_t st);
cudaError_t mask_mark_budget(uint8_t* mask, int nx, int ny, int nz, cudaStream_t st);
// Ordered list of the cells whose mask has a given bit (the near-solid cells, the budget cells): per-chunk
// counts, then (after a host-side exclusive scan into offsets) the cell indices in ascending order.
constexpr int kListChunk = 1024;
cudaError_t mask_list_counts(const uint8_t* mask, size_t n, uint8_t bit, int* chunk_counts, cudaStream_t st);
cudaError_t mask_list_fill(const uint8_t* mask, size_t n, uint8_t bit, const int* chunk_offsets, int* list,
                           cudaStream_t st);

}  // namespace vf
