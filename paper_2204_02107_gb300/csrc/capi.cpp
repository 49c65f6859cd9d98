// Step engine and C ABI of the ventilation-flow library (declared in include/ventflow.h).
//
// A grid owns every device buffer of one room: the state q = (u, v, w, c), three RK4 stage states (q2, q3, q4 in
// the buffers qa, qb, acc; no accumulator is carried between stages), the pressure p / rho (kept between steps as the warm start of Eq. 9; the paper's p carries a factor
// dt, so the solver works on D u* / dt and the projection subtracts dt G p), the divergence r, the half
// spectrum, a staging buffer for host/device transfers, the packed mask and the FFT tables.  A step is a fixed
// sequence of kernel launches on the grid's stream; it is captured once into a CUDA graph and replayed.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_plan.h"
#include "grid.h"

using vf::FftAxis;
using vf::FlowConsts;
using vf::Kernels;
using vf::PoissonArgs;
using vf::StageArgs;

namespace {

const char* kStatusNames[] = {"VF_OK", "VF_EINVAL", "VF_ESIZE", "VF_ENOMEM", "VF_ECUDA", "VF_ESTATE",
                              "VF_ENONFINITE", "VF_ETIMEOUT"};

int set_err(vf_grid* g, int code, const std::string& msg)
{
    if (g) g->err = msg;
    return code;
}

int fail_cuda(vf_grid* g, cudaError_t e, const char* what)
{
    if (g) {
        g->status = VF_ECUDA;
        g->err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return VF_ECUDA;
}

#define VF_CK(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return fail_cuda(g, e_, #call);       \
    } while (0)

// Largest grid: cell indices and the index arithmetic of the kernels (offsets of up to a few thousand cells past
// an index) stay far inside 32-bit integers.
constexpr long long kMaxCells = 1LL << 30;

bool smooth235_even(int n)
{
    if (n < 8 || n % 2) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

void* galloc(vf_grid* g, size_t bytes)
{
    ++g->alloc_count;
    if (g->fail_alloc_at > 0 && g->alloc_count == g->fail_alloc_at) return nullptr;
    void* p = nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (g->have_alloc) {
        p = g->alloc.alloc(bytes, (void*)g->stream, g->alloc.ctx);
    } else if (cudaMallocAsync(&p, bytes, g->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        g->allocs.push_back(p);
        g->bytes += bytes;
        if (cudaMemsetAsync(p, 0, bytes, g->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    return p;
}

void free_particles(vf_grid* g)
{
    if (g->particle_buf) {
        if (g->have_alloc) g->alloc.free(g->particle_buf, (void*)g->stream, g->alloc.ctx);
        else cudaFreeAsync(g->particle_buf, g->stream);
        g->bytes -= g->particle_bytes;
    }
    g->particle_buf = nullptr;
    g->particle_bytes = 0;
    g->particles.n = 0;
}

void release_all(vf_grid* g)
{
    for (int i = 0; i < 4; ++i)
        if (g->gexec[i]) { cudaGraphExecDestroy(g->gexec[i]); g->gexec[i] = nullptr; }
    g->graph_ok = false;
    free_particles(g);
    for (void* p : g->allocs) {
        if (g->have_alloc) g->alloc.free(p, (void*)g->stream, g->alloc.ctx);
        else cudaFreeAsync(p, g->stream);
    }
    g->allocs.clear();
    if (g->stream) cudaStreamSynchronize(g->stream);
}

template <typename T>
FlowConsts<T> flow_consts(const vf_grid* g)
{
    FlowConsts<T> k{};
    const vf_grid_desc& d = g->d;
    k.nx = d.nx; k.ny = d.ny; k.nz = d.nz;
    for (int i = 0; i < vf::kZcKinds; ++i) k.zc[i] = g->zc[i];
    const double h[3] = {d.lx / d.nx, d.ly / d.ny, d.lz / d.nz};
    for (int j = 0; j < 3; ++j) {
        k.i2h[j] = (T)(1.0 / (2.0 * h[j]));
        k.i2h_div[j] = (T)(1.0 / (2.0 * h[j] * d.dt));
        k.i2h_dt[j] = (T)(d.dt / (2.0 * h[j]));
        k.q4h[j] = (T)(1.0 / (4.0 * h[j]));
        k.ih[j] = (T)(1.0 / h[j]);
        k.ih2[j] = (T)(1.0 / (h[j] * h[j]));
        k.bf[j] = (T)d.body_force[j];
        k.uset[j] = g->has_target ? T(0) : (T)g->uset[j];
    }
    const double tau = d.tau_f > 0 ? d.tau_f : d.dt;
    k.nu = (T)d.nu;
    k.alpha = (T)(d.alpha_c < 0 ? d.nu : d.alpha_c);
    k.inv_tau = (T)(1.0 / tau);
    k.dt = (T)d.dt;
    k.dt2 = (T)(d.dt / 2.0);
    k.dt3 = (T)(d.dt / 3.0);
    k.dt6 = (T)(d.dt / 6.0);
    k.third = (T)(1.0 / 3.0);
    k.cset = g->has_target ? T(0) : (T)g->cset;
    k.filt = (T)(1.0 / std::pow(M_PI, 6));
    k.dyn = g->dynamic ? g->dtctl : nullptr;
    return k;
}

template <typename T>
PoissonArgs<T> poisson_args(const vf_grid* g, T* f, T* p, int use_mask)
{
    PoissonArgs<T> a{};
    const vf_grid_desc& d = g->d;
    a.nx = d.nx; a.ny = d.ny; a.nz = d.nz; a.M = d.nx / 2;
    a.f = f; a.p = p; a.smask = g->smask;
    a.near_list = g->near_list;
    a.near_r = (T*)g->near_r;
    a.n_near = use_mask ? g->n_near : 0;
    a.plane_layout = g->plane_layout ? 1 : 0;
    a.reg = g->reg;
    a.rx = g->reg_rx; a.ry = g->reg_ry; a.rz = g->reg_rz;
    a.gx = g->reg_gx; a.gy = g->reg_gy; a.gz = g->reg_gz;
    a.reg_sp = g->reg_sp; a.reg_spx = g->reg_spx; a.reg_sb = g->reg_sb;
    a.reg_tile = g->reg_tile; a.reg_sy = g->reg_sy; a.reg_tb = g->reg_tb; a.reg_st = g->reg_st;
    a.spec = g->spec;
    a.twx = g->twx; a.twy = g->twy; a.twz = g->twz; a.twr = g->twr;
    a.lamx = (const T*)g->lamx; a.lamy = (const T*)g->lamy; a.lamz = (const T*)g->lamz;
    a.krev_y = g->krev_y; a.krev_z = g->krev_z;
    const double h[3] = {d.lx / d.nx, d.ly / d.ny, d.lz / d.nz};
    for (int j = 0; j < 3; ++j) a.i2h2[j] = (T)(1.0 / (4.0 * h[j] * h[j]));
    a.invN = (T)(1.0 / ((double)d.nx * d.ny * d.nz));
    a.ax = g->ax; a.ay = g->ay; a.az = g->az;
    a.ny_div = vf::make_fast_div((uint32_t)d.ny);
    a.nx_div = vf::make_fast_div((uint32_t)d.nx);
    a.rows_per_block = g->rows_per_block;
    a.cols_per_block = g->cols_per_block;
    return a;
}

vf::ReduceArgsDev reduce_args(const vf_grid* g)
{
    vf::ReduceArgsDev r{};
    r.partial = g->red_partial;
    r.div_partial = g->div_partial;
    r.hist_accum = g->hist_accum;
    r.done = g->red_done;
    r.out = g->red_out;
    r.history = g->history;
    r.hist_count = g->dev_counters;
    r.step_counter = g->dev_counters + 1;
    r.nonfinite = g->nonfinite;
    r.history_capacity = g->d.history_capacity;
    r.dV = (g->d.lx / g->d.nx) * (g->d.ly / g->d.ny) * (g->d.lz / g->d.nz);
    r.dt = g->d.dt;
    r.t0 = g->t0;
    r.dyn = g->dynamic ? g->dtctl : nullptr;
    return r;
}

// Budget CTAs of a recorded step's stage 3 and 4 launches: about one CTA per 256 (cell, stage state) items, at
// least one, at most one z slice of the stage grid.
template <typename T>
vf::BudgetArgs budget_args(const vf_grid* g, const FlowConsts<T>& k)
{
    const vf_grid_desc& d = g->d;
    vf::BudgetArgs b{};
    b.n = g->n_budget;
    b.cap = Kernels<T>::budget_cta_capacity(k);
    b.ctas = (int)std::min<long long>(b.cap, std::max<long long>(1, (2LL * g->n_budget + 255) / 256));
    b.list = g->budget_list;
    b.partial = g->budget_partial;
    b.done = g->budget_done;
    b.out = g->budget_out;
    const double h[3] = {d.lx / d.nx, d.ly / d.ny, d.lz / d.nz};
    b.dV = h[0] * h[1] * h[2];
    b.dt = d.dt;
    b.inv_tau = 1.0 / (d.tau_f > 0 ? d.tau_f : d.dt);
    b.alpha = d.alpha_c < 0 ? d.nu : d.alpha_c;
    b.cset = g->cset;
    for (int j = 0; j < 3; ++j) b.ih[j] = 1.0 / h[j];
    return b;
}

// Ordered list of the cells whose mask has `bit`: per-chunk counts, host exclusive scan, fill (synchronous).
cudaError_t cell_list(vf_grid* g, uint8_t bit, int* list, int* count)
{
    const size_t chunks = (g->N + vf::kListChunk - 1) / vf::kListChunk;
    int* d_counts = (int*)g->staging;
    cudaError_t e;
    if ((e = vf::mask_list_counts(g->mask, g->N, bit, d_counts, g->stream)) != cudaSuccess) return e;
    std::vector<int> counts(chunks);
    if ((e = cudaMemcpyAsync(counts.data(), d_counts, chunks * sizeof(int), cudaMemcpyDeviceToHost, g->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
        return e;
    int total = 0;
    for (size_t c = 0; c < chunks; ++c) {
        const int n = counts[c];
        counts[c] = total;
        total += n;
    }
    if ((e = cudaMemcpyAsync(d_counts, counts.data(), chunks * sizeof(int), cudaMemcpyHostToDevice, g->stream)) !=
            cudaSuccess ||
        (e = vf::mask_list_fill(g->mask, g->N, bit, d_counts, list, g->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(g->stream)) != cudaSuccess)
        return e;
    *count = total;
    return cudaSuccess;
}

void drop_graphs(vf_grid* g);

// The budget bit of every cell (from beta, S and the room bits) and the list of those cells; the step graphs
// carry the list's length, so they are rebuilt.
cudaError_t budget_cells(vf_grid* g)
{
    cudaError_t e = vf::mask_mark_budget(g->mask, g->d.nx, g->d.ny, g->d.nz, g->stream);
    if (e == cudaSuccess) e = cell_list(g, vf::kBitBudget, g->budget_list, &g->n_budget);
    if (e == cudaSuccess) drop_graphs(g);
    return e;
}

int pressure_iters(const vf_grid* g)
{
    if (g->d.n_pressure_iters <= 0) return 0;
    return g->has_solid ? g->d.n_pressure_iters : 1;
}

// The reduction record of the grid's current state (the step that just ended): the flat reduction of the filtered
// state with the filter's records, or the standalone reduction when the filter is off.
template <typename T>
cudaError_t enqueue_reduction_t(vf_grid* g, cudaStream_t st)
{
    const FlowConsts<T> k = flow_consts<T>(g);
    vf::ReduceArgsDev ra = reduce_args(g);
    ra.budget = g->budget_out;
    if (g->d.filter) {
        ra.filter_budget = 1;
        return Kernels<T>::reduce_state(g->q, g->mask, k, ra, 1, g->nred, st);
    }
    return Kernels<T>::reduce(g->q, g->mask, k, ra, 1, st);
}

cudaError_t enqueue_reduction(vf_grid* g, cudaStream_t st)
{
    return g->fp64 ? enqueue_reduction_t<double>(g, st) : enqueue_reduction_t<float>(g, st);
}

// Step launches.  with_reduce: this step writes a reduction record (budget CTAs in stages 3 and 4, the filter's
// records); lag: its reduction kernel is not launched here but by the next step (reduce_prev) or a flush.
// reduce_prev: the previous step's record is reduced on the side stream while stages 1 and 2 run (they write
// only the stage states qa and qb; the reduction reads q, the filter's records and the budget terms, which nothing
// before stage 3 writes), joined before stage 3.  Not with a dynamic time step, whose adjust kernel rewrites the
// time the record reads.
template <typename T>
cudaError_t enqueue_step_t(vf_grid* g, cudaStream_t st, bool with_reduce, const vf::LaunchHook* hook, bool lag = false,
                           bool reduce_prev = false)
{
    auto mark = [&](int phase) { if (hook) (*hook)(phase); };
    const FlowConsts<T> k = flow_consts<T>(g);
    cudaError_t e;
    // dynamic time step: dt of this step from the Courant rate of the state it starts from (device side)
    unsigned long long* sigma_out = g->dynamic ? &g->dtctl->sigma_bits : nullptr;
    if (g->dynamic) {
        if ((e = vf::adjust_dt(g->dtctl, st)) != cudaSuccess) return e;
        mark(VF_PHASE_ADJUST_DT);
    }
    if (reduce_prev) {
        if (g->dynamic) return cudaErrorInvalidValue;
        if ((e = cudaEventRecord(g->ev_fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(g->side_stream, g->ev_fork, 0)) != cudaSuccess ||
            (e = enqueue_reduction_t<T>(g, g->side_stream)) != cudaSuccess ||
            (e = cudaEventRecord(g->ev_join, g->side_stream)) != cudaSuccess)
            return e;
    }
    StageArgs<T> a{};
    a.mask = g->mask;
    a.smask = g->smask;
    a.sval = g->smooth_s ? (const T*)g->sval : nullptr;
    a.target = g->has_target ? g->target : nullptr;
    a.qn = g->q;
    // stage states: q2 in qa, q3 in qb, q4 in acc; stage 4 writes q* over q2 (each cell reads its own q2 first)
    a.qs = g->q; a.out = g->qa;
    if ((e = Kernels<T>::stage(1, a, k, st)) != cudaSuccess) return e;
    mark(VF_PHASE_STAGE1);
    a.qs = g->qa; a.out = g->qb;
    if ((e = Kernels<T>::stage(2, a, k, st)) != cudaSuccess) return e;
    mark(VF_PHASE_STAGE2);
    a.qs = g->qb; a.out = g->acc;
    if (reduce_prev && (e = cudaStreamWaitEvent(st, g->ev_join, 0)) != cudaSuccess) return e;
    if (with_reduce) {
        // scalar budget: extra CTAs of stage 3 read q_n and q2, those of stage 4 q3 and q4 (none is written by
        // the launch that reads it)
        a.bud = budget_args(g, k);
        a.bud.slot = 0;
        a.bud.qa = g->q; a.bud.wa = 1.0 / 6.0;
        a.bud.qb = g->qa; a.bud.wb = 1.0 / 3.0;
    }
    if ((e = Kernels<T>::stage(3, a, k, st)) != cudaSuccess) return e;
    mark(VF_PHASE_STAGE3);
    if (with_reduce) {
        a.bud.ctas_prev = a.bud.ctas;
        a.bud.slot = 1;
        a.bud.qa = g->qb; a.bud.wa = 1.0 / 3.0;
        a.bud.qb = g->acc; a.bud.wb = 1.0 / 6.0;
    }
    a.qs = g->acc; a.q2 = g->qa; a.q3 = g->qb; a.out = g->qa;
    if ((e = Kernels<T>::stage(4, a, k, st)) != cudaSuccess) return e;
    mark(VF_PHASE_STAGE4);
    void* qstar = g->qa;
    const int iters = pressure_iters(g);
    if (iters > 0) {
        if ((e = Kernels<T>::divergence(qstar, (T*)g->f, k, st)) != cudaSuccess) return e;
        mark(VF_PHASE_DIV);
        const PoissonArgs<T> pa = poisson_args<T>(g, (T*)g->f, (T*)g->p, g->has_solid ? 1 : 0);
        for (int it = 0; it < iters; ++it)
            if ((e = Kernels<T>::poisson_iteration(pa, it == 0, st, hook)) != cudaSuccess) return e;
    }
    long long* step_counter = g->dev_counters + 1;
    // projection into qb (then filtered into q) or straight into q
    void* proj_out = g->d.filter ? g->qb : g->q;
    if ((e = Kernels<T>::project(qstar, (const T*)g->p, proj_out, g->mask, step_counter, k, st,
                                 g->d.filter ? nullptr : sigma_out)) != cudaSuccess)
        return e;
    mark(VF_PHASE_PROJECT);
    if (g->d.filter) {
        // with the filter on, the filter records the divergence of its input (the projected velocity) and the
        // flat reduction of the filtered state follows
        vf::ReduceArgsDev ra = reduce_args(g);
        ra.budget = g->budget_out;
        ra.filter_budget = 1;
        if ((e = Kernels<T>::filter(g->qb, g->q, g->mask, k, with_reduce ? &ra : nullptr, st, sigma_out)) !=
            cudaSuccess)
            return e;
        mark(VF_PHASE_FILTER);
    }
    if (with_reduce && !lag) {
        if ((e = enqueue_reduction_t<T>(g, st)) != cudaSuccess) return e;
        mark(VF_PHASE_REDUCE);
    }
    if (g->particles.n > 0) {
        vf::ParticleArgs P = g->particles;
        P.dyn = g->dynamic ? g->dtctl : nullptr;
        if ((e = vf::advance_particles<T>(P, g->q, g->mask, st)) != cudaSuccess) return e;
        mark(VF_PHASE_PARTICLES);
    }
    return cudaSuccess;
}

cudaError_t enqueue_step(vf_grid* g, cudaStream_t st, bool with_reduce, const vf::LaunchHook* hook = nullptr,
                         bool lag = false, bool reduce_prev = false)
{
    return g->fp64 ? enqueue_step_t<double>(g, st, with_reduce, hook, lag, reduce_prev)
                   : enqueue_step_t<float>(g, st, with_reduce, hook, lag, reduce_prev);
}

// Event recorder behind vf_profile_steps: one event after every launch, tagged with its phase.
struct PhaseRecorder {
    cudaStream_t stream;
    std::vector<cudaEvent_t> events;
    std::vector<int> phases;
    cudaError_t err = cudaSuccess;
    static void hook(void* ctx, int phase)
    {
        PhaseRecorder* r = (PhaseRecorder*)ctx;
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e == cudaSuccess) e = cudaEventRecord(ev, r->stream);
        if (e != cudaSuccess) { r->err = e; return; }
        r->events.push_back(ev);
        r->phases.push_back(phase);
    }
};

void drop_graphs(vf_grid* g)
{
    for (int i = 0; i < 4; ++i)
        if (g->gexec[i]) { cudaGraphExecDestroy(g->gexec[i]); g->gexec[i] = nullptr; }
    g->graph_ok = false;
}

// Step graphs: variant bit 0 = the step writes a record, bit 1 = the previous step's record is reduced alongside
// stages 1-2 (the record of a recorded step is then left to the next step or a flush: lagged).  Variants 2 and 3
// exist only for a fixed time step.
int capture_graphs(vf_grid* g)
{
    drop_graphs(g);
    for (int i = 0; i < 4; ++i) {
        if (i >= 2 && g->dynamic) continue;
        cudaGraph_t graph = nullptr;
        VF_CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
        const bool lagged = !g->dynamic;
        cudaError_t e = enqueue_step(g, g->cap_stream, (i & 1) != 0, nullptr, lagged && (i & 1), (i & 2) != 0);
        cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail_cuda(g, e, "capture step"); }
        if (e2 != cudaSuccess) return fail_cuda(g, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g->gexec[i], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail_cuda(g, e, "cudaGraphInstantiate");
    }
    g->graph_ok = true;
    return VF_OK;
}

template <typename T>
int build_tables_t(vf_grid* g)
{
    const vf_grid_desc& d = g->d;
    const int M = d.nx / 2;
    struct C2 { T x, y; };
    auto roots = [](int n, int count) {
        std::vector<C2> t(count);
        for (int m = 0; m < count; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)n;
            t[m].x = (T)std::cos(a);
            t[m].y = (T)(-std::sin(a));
        }
        return t;
    };
    auto lam = [](int n, int count, double h) {
        std::vector<T> t(count);
        for (int k = 0; k < count; ++k) {
            const double s = (k == 0 || 2 * k == n) ? 0.0 : std::sin(2.0 * M_PI * (double)k / (double)n);
            t[k] = (T)(s * s / (h * h));
        }
        return t;
    };
    const std::vector<C2> tx = roots(M, M), ty = roots(d.ny, d.ny), tz = roots(d.nz, d.nz), tr = roots(d.nx, M + 1);
    const std::vector<T> lx = lam(d.nx, M, d.lx / d.nx), ly = lam(d.ny, d.ny, d.ly / d.ny),
                         lz = lam(d.nz, d.nz, d.lz / d.nz);
    std::vector<int> ry(d.ny), rz(d.nz);
    vf::digit_reversal(g->ay, ry.data());
    vf::digit_reversal(g->az, rz.data());
    struct Up { void** dst; const void* src; size_t bytes; };
    const Up ups[] = {{&g->twx, tx.data(), tx.size() * sizeof(C2)}, {&g->twy, ty.data(), ty.size() * sizeof(C2)},
                      {&g->twz, tz.data(), tz.size() * sizeof(C2)}, {&g->twr, tr.data(), tr.size() * sizeof(C2)},
                      {&g->lamx, lx.data(), lx.size() * sizeof(T)}, {&g->lamy, ly.data(), ly.size() * sizeof(T)},
                      {&g->lamz, lz.data(), lz.size() * sizeof(T)},
                      {(void**)&g->krev_y, ry.data(), ry.size() * sizeof(int)},
                      {(void**)&g->krev_z, rz.data(), rz.size() * sizeof(int)}};
    for (const Up& u : ups) {
        *u.dst = galloc(g, u.bytes);
        if (!*u.dst) return set_err(g, VF_ENOMEM, "table allocation failed");
        VF_CK(cudaMemcpyAsync(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, g->stream));
    }
    VF_CK(cudaStreamSynchronize(g->stream));   // host vectors die here
    // the register path keeps the spectrum plane by plane ([kx][z][y]) whether or not a plane fits in shared memory;
    // the generic path uses that layout only with its whole-plane kernel (VF_TILE_FFT / VF_GENERIC_FFT: generic)
    const bool generic = std::getenv("VF_TILE_FFT") || std::getenv("VF_GENERIC_FFT");
    if (!generic && vf::RegFft<T>::eligible(d.nx, d.ny, d.nz)) {
        g->plane_layout = true;
        PoissonArgs<T> ra = poisson_args<T>(g, nullptr, nullptr, 0);
        vf::RegFft<T>::configure(ra);
        g->reg = ra.reg;
        g->reg_rx = ra.rx; g->reg_ry = ra.ry; g->reg_rz = ra.rz;
        g->reg_gx = ra.gx; g->reg_gy = ra.gy; g->reg_gz = ra.gz;
        g->reg_sp = ra.reg_sp; g->reg_spx = ra.reg_spx; g->reg_sb = ra.reg_sb;
        g->reg_tile = ra.reg_tile; g->reg_sy = ra.reg_sy; g->reg_tb = ra.reg_tb; g->reg_st = ra.reg_st;
    } else {
        g->plane_layout = Kernels<T>::plane_fits(d.ny, d.nz) && !std::getenv("VF_TILE_FFT");
    }
    const PoissonArgs<T> pa = poisson_args<T>(g, nullptr, nullptr, 0);
    VF_CK(Kernels<T>::poisson_prepare(pa));
    return VF_OK;
}

int check(const vf_grid* g)
{
    if (!g) return VF_EINVAL;
    return g->status;
}

// Copy `bytes` from the caller (host or device) into device memory the grid can read, returning the pointer.
const void* stage_input(vf_grid* g, const void* src, size_t bytes, int mem, int* rc)
{
    *rc = VF_OK;
    if (mem == VF_DEVICE) return src;
    cudaError_t e = cudaMemcpyAsync(g->staging, src, bytes, cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) { *rc = fail_cuda(g, e, "cudaMemcpyAsync(staging)"); return nullptr; }
    return g->staging;
}

template <typename T>
cudaError_t mask_fields(vf_grid* g)
{
    return Kernels<T>::apply_mask(g->q, g->mask, g->N, g->stream);
}

// Lengths of the three FFT axes: the x half length nx/2, ny, nz.
void fft_lengths(const vf_grid* g, int len[3])
{
    len[0] = g->d.nx / 2;
    len[1] = g->d.ny;
    len[2] = g->d.nz;
}

// Every index names a candidate schedule of its axis length.
bool fft_indices_valid(const vf_grid* g, const int idx[3])
{
    int len[3];
    fft_lengths(g, len);
    for (int a = 0; a < 3; ++a)
        if (idx[a] < 0 || idx[a] >= (int)vf::fft_schedules(len[a]).size()) return false;
    return true;
}

// Switch the generic FFT passes to the schedules idx (valid indices): rebuild the three axes and, once the tables
// exist, the digit-reversal tables of the in-place y and z transforms (same sizes, copied over the old ones).  The
// step graphs are dropped.  Stream-ordered copies; waits for them, since the host tables die here.
int set_fft_sched(vf_grid* g, const int idx[3])
{
    int len[3];
    fft_lengths(g, len);
    for (int a = 0; a < 3; ++a) g->fft_sched[a] = idx[a];
    g->ax = vf::make_fft_axis_sched(len[0], idx[0]);
    g->ay = vf::make_fft_axis_sched(len[1], idx[1]);
    g->az = vf::make_fft_axis_sched(len[2], idx[2]);
    drop_graphs(g);
    if (!g->krev_y || !g->krev_z) return VF_OK;
    std::vector<int> ry(g->d.ny), rz(g->d.nz);
    vf::digit_reversal(g->ay, ry.data());
    vf::digit_reversal(g->az, rz.data());
    VF_CK(cudaMemcpyAsync(g->krev_y, ry.data(), ry.size() * sizeof(int), cudaMemcpyHostToDevice, g->stream));
    VF_CK(cudaMemcpyAsync(g->krev_z, rz.data(), rz.size() * sizeof(int), cudaMemcpyHostToDevice, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

}  // namespace

namespace vf_engine {

cudaError_t refresh_sigma(vf_grid* g, cudaStream_t st)
{
    if (!g->dynamic || !g->sigma_stale) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(&g->dtctl->sigma_bits, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = g->fp64 ? Kernels<double>::courant_rate(g->q, flow_consts<double>(g), g->N, &g->dtctl->sigma_bits, st)
                    : Kernels<float>::courant_rate(g->q, flow_consts<float>(g), g->N, &g->dtctl->sigma_bits, st);
    if (e == cudaSuccess) g->sigma_stale = false;
    return e;
}

cudaError_t enqueue_step(vf_grid* g, cudaStream_t st, bool with_reduce)
{
    return ::enqueue_step(g, st, with_reduce);
}

size_t grid_bytes(const vf_grid_desc& d)
{
    auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t esz = d.precision == VF_FP64 ? 8 : 4, cpx = 2 * esz;
    const size_t N = (size_t)d.nx * d.ny * d.nz, M = (size_t)d.nx / 2;
    FlowConsts<float> k{};
    k.nx = d.nx; k.ny = d.ny; k.nz = d.nz;
    const size_t nred = (size_t)Kernels<float>::reduce_blocks(k);
    k.zc[vf::kZcFilter] = vf::kZChunkMin;
    const size_t ndiv = (size_t)Kernels<float>::filter_warps(k);
    size_t b = 4 * r256(4 * N * esz) + 5 * r256(N * esz) + r256(N * 4) + r256(N * 8) + 2 * r256(N);
    b += r256(nred * vf::kRedSlots * 8) + r256(ndiv * vf::kDivRecord * 8) + r256((vf::kHistBins + 2) * 8) + r256(4) +
         r256(sizeof(vf_reduce));
    b += r256((size_t)d.history_capacity * sizeof(vf_reduce)) + r256(16) + r256(4) + r256(8);
    b += r256(sizeof(vf::DtCtl)) + r256(3 * sizeof(double));
    b += r256(2 * (size_t)Kernels<float>::budget_cta_capacity(k) * vf::kBudgetTerms * 8) + r256(N * 4) + r256(4) +
         r256(vf::kBudgetTerms * 8);
    b += r256(M * cpx) + r256(d.ny * cpx) + r256(d.nz * cpx) + r256((M + 1) * cpx);
    b += r256(M * esz) + r256(d.ny * esz) + r256(d.nz * esz) + r256(d.ny * 4) + r256(d.nz * 4);
    return b;
}

}  // namespace vf_engine

extern "C" {

int64_t vf_grid_bytes(const vf_grid_desc* d)
{
    if (!d) return -1;
    return (int64_t)vf_engine::grid_bytes(*d);
}


int vf_grid_desc_default(vf_grid_desc* d)
{
    if (!d) return VF_EINVAL;
    std::memset(d, 0, sizeof(*d));
    d->nx = d->ny = d->nz = 64;
    d->lx = d->ly = d->lz = 1.0;
    d->nu = 1.6e-5;
    d->alpha_c = -1.0;
    d->dt = 1e-3;
    d->tau_f = 0.0;
    d->n_pressure_iters = 4;
    d->filter = 1;
    d->precision = VF_FP32_MIXED;
    d->history_capacity = 4096;
    d->cuda_stream = nullptr;
    d->alloc = nullptr;
    return VF_OK;
}

int vf_create_grid(const vf_grid_desc* d, vf_grid** out)
{
    if (!d || !out) return VF_EINVAL;
    *out = nullptr;
    if (!smooth235_even(d->nx) || !smooth235_even(d->ny) || !smooth235_even(d->nz)) return VF_ESIZE;
    if (!(d->lx > 0) || !(d->ly > 0) || !(d->lz > 0) || !(d->dt > 0) || !(d->nu >= 0)) return VF_EINVAL;
    if (d->precision != VF_FP64 && d->precision != VF_FP32_MIXED) return VF_EINVAL;
    if (d->n_pressure_iters < 0 || d->history_capacity < 1) return VF_EINVAL;
    if (!(d->courant_max >= 0.0)) return VF_EINVAL;
    if ((long long)d->nx * d->ny * d->nz > kMaxCells) return VF_ESIZE;

    vf_grid* g = new vf_grid();
    g->d = *d;
    g->fp64 = d->precision == VF_FP64;
    g->esz = g->fp64 ? 8 : 4;
    g->N = (size_t)d->nx * d->ny * d->nz;
    if (d->alloc) { g->alloc = *d->alloc; g->have_alloc = g->alloc.alloc && g->alloc.free; }
    if (const char* s = std::getenv("VF_FAULT_ALLOC_AT")) g->fail_alloc_at = std::atoi(s);
    if (std::getenv("VF_NO_GRAPH")) g->use_graph = false;

    auto fail = [&](int code) {
        release_all(g);
        if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
        if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
        if (g->side_stream) cudaStreamDestroy(g->side_stream);
        if (g->ev_fork) cudaEventDestroy(g->ev_fork);
        if (g->ev_join) cudaEventDestroy(g->ev_join);
        delete g;
        return code;
    };
    if (d->cuda_stream) {
        g->stream = (cudaStream_t)d->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(VF_ECUDA);
        g->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(VF_ECUDA);
    if (cudaStreamCreateWithFlags(&g->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(VF_ECUDA);

    const int M = d->nx / 2;
    {
        // the FFT passes keep up to three tiles of their batch and a twiddle table in shared memory (at most
        // 227 KB per CTA): ny, nz <= 592 in FP32 and <= 581 in FP64
        const size_t cplx = g->fp64 ? 16 : 8, tb = g->fp64 ? 8 : 16, limit = 227 * 1024;
        const size_t n = (size_t)std::max(d->ny, d->nz);
        if ((3 * tb * n + n) * cplx > limit || 4 * (size_t)M * cplx > limit) return fail(VF_ESIZE);
    }
    g->ax = vf::make_fft_axis(M);
    g->ay = vf::make_fft_axis(d->ny);
    g->az = vf::make_fft_axis(d->nz);
    const int target = g->fp64 ? 1024 : 2048;   // complex values per CTA in the x passes
    g->rows_per_block = std::max(1, target / M);
    g->cols_per_block = g->fp64 ? 8 : 16;

    const size_t fb = g->N * g->esz;
    void** states[] = {&g->q, &g->acc, &g->qa, &g->qb};
    for (void** f : states)
        if (!(*f = galloc(g, 4 * fb))) return fail(VF_ENOMEM);
    void** scalars[] = {&g->p, &g->f, &g->spec, &g->near_r, &g->sval};
    for (void** f : scalars)
        if (!(*f = galloc(g, fb))) return fail(VF_ENOMEM);
    if (!(g->near_list = (int*)galloc(g, g->N * sizeof(int)))) return fail(VF_ENOMEM);
    if (!(g->staging = galloc(g, g->N * 8))) return fail(VF_ENOMEM);
    if (!(g->mask = (uint8_t*)galloc(g, g->N))) return fail(VF_ENOMEM);
    if (!(g->smask = (uint8_t*)galloc(g, g->N))) return fail(VF_ENOMEM);

    {
        vf_tiles t{};
        if (vf_tile_cache_lookup(d->nx, d->ny, d->nz, d->precision, &t) == 1) {
            g->zc[0] = t.zc_stage; g->zc[1] = t.zc_div; g->zc[2] = t.zc_project; g->zc[3] = t.zc_filter;
            const int idx[3] = {t.fft_x, t.fft_y, t.fft_z};
            if (fft_indices_valid(g, idx)) {
                for (int a = 0; a < 3; ++a) g->fft_sched[a] = idx[a];
                g->ax = vf::make_fft_axis_sched(M, idx[0]);
                g->ay = vf::make_fft_axis_sched(d->ny, idx[1]);
                g->az = vf::make_fft_axis_sched(d->nz, idx[2]);
            }
        }
    }
    const FlowConsts<float> kf = flow_consts<float>(g);
    g->nred = Kernels<float>::reduce_blocks(kf);   // enough partial slots for the smallest filter chunk
    if (!(g->red_partial = (double*)galloc(g, (size_t)g->nred * vf::kRedSlots * sizeof(double)))) return fail(VF_ENOMEM);
    {
        FlowConsts<float> kmin = kf;   // the filter's divergence records under its smallest chunk
        kmin.zc[vf::kZcFilter] = vf::kZChunkMin;
        g->ndiv = Kernels<float>::filter_warps(kmin);
    }
    if (!(g->div_partial = (double*)galloc(g, (size_t)g->ndiv * vf::kDivRecord * sizeof(double))))
        return fail(VF_ENOMEM);
    if (!(g->hist_accum = (unsigned long long*)galloc(g, (vf::kHistBins + 2) * sizeof(unsigned long long))))
        return fail(VF_ENOMEM);
    if (!(g->red_done = (unsigned int*)galloc(g, sizeof(unsigned int)))) return fail(VF_ENOMEM);
    if (!(g->red_out = (vf_reduce*)galloc(g, sizeof(vf_reduce)))) return fail(VF_ENOMEM);
    if (!(g->history = (vf_reduce*)galloc(g, (size_t)d->history_capacity * sizeof(vf_reduce)))) return fail(VF_ENOMEM);
    if (!(g->dev_counters = (long long*)galloc(g, 2 * sizeof(long long)))) return fail(VF_ENOMEM);
    if (!(g->nonfinite = (int*)galloc(g, sizeof(int)))) return fail(VF_ENOMEM);
    if (!(g->solid_count = (unsigned long long*)galloc(g, sizeof(unsigned long long)))) return fail(VF_ENOMEM);
    if (!(g->dtctl = (vf::DtCtl*)galloc(g, sizeof(vf::DtCtl)))) return fail(VF_ENOMEM);
    if (!(g->force_acc = (double*)galloc(g, 3 * sizeof(double)))) return fail(VF_ENOMEM);
    if (!(g->budget_partial = (double*)galloc(g, 2 * (size_t)Kernels<float>::budget_cta_capacity(kf) *
                                                     vf::kBudgetTerms * sizeof(double))))
        return fail(VF_ENOMEM);
    if (!(g->budget_list = (int*)galloc(g, g->N * sizeof(int)))) return fail(VF_ENOMEM);
    if (!(g->budget_done = (unsigned int*)galloc(g, sizeof(unsigned int)))) return fail(VF_ENOMEM);
    if (!(g->budget_out = (double*)galloc(g, vf::kBudgetTerms * sizeof(double)))) return fail(VF_ENOMEM);
    {
        // the control block starts at the given dt (constants with the same formulas as the adjust kernel)
        g->dynamic = d->courant_max > 0.0;
        vf::DtCtl c{};
        c.dt = d->dt;
        c.t_end = 0.0;
        c.dt2 = d->dt / 2.0;
        c.dt3 = d->dt / 3.0;
        c.dt6 = d->dt / 6.0;
        c.inv_tau = 1.0 / (d->tau_f > 0.0 ? d->tau_f : d->dt);
        const double h[3] = {d->lx / d->nx, d->ly / d->ny, d->lz / d->nz};
        for (int j = 0; j < 3; ++j) {
            c.h[j] = h[j];
            c.i2h_div[j] = 1.0 / (2.0 * h[j] * d->dt);
            c.i2h_dt[j] = d->dt / (2.0 * h[j]);
        }
        c.sigma_bits = 0ull;
        c.courant_max = d->courant_max;
        c.dt_max = d->dt;
        c.tau_f = d->tau_f;
        if (cudaMemcpyAsync(g->dtctl, &c, sizeof(c), cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
            cudaStreamSynchronize(g->stream) != cudaSuccess)
            return fail(VF_ECUDA);
    }

    int rc = g->fp64 ? build_tables_t<double>(g) : build_tables_t<float>(g);
    if (rc != VF_OK) return fail(rc == VF_ECUDA ? VF_ECUDA : rc);
    // all-fluid mask, every cell in the room region
    if (vf::mask_fill(g->mask, vf::kBitBeta | vf::kBitRoom, g->N, g->stream) != cudaSuccess) return fail(VF_ECUDA);
    if (vf::build_stencil_mask(g->mask, g->smask, d->nx, d->ny, d->nz, g->stream) != cudaSuccess) return fail(VF_ECUDA);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return fail(VF_ECUDA);
    *out = g;
    return VF_OK;
}

int vf_destroy(vf_grid* g)
{
    if (!g) return VF_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    release_all(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->side_stream) cudaStreamDestroy(g->side_stream);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
    return VF_OK;
}

int vf_set_mask(vf_grid* g, const uint8_t* beta, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!beta || (mem != VF_HOST && mem != VF_DEVICE)) return set_err(g, VF_EINVAL, "vf_set_mask: bad argument");
    const void* src = stage_input(g, beta, g->N, mem, &rc);
    if (rc) return rc;
    VF_CK(vf::mask_merge(g->mask, (const uint8_t*)src, vf::kBitBeta, g->N, g->stream));
    VF_CK(vf::mask_mark_near_solid(g->mask, g->d.nx, g->d.ny, g->d.nz, g->stream));
    VF_CK(g->fp64 ? mask_fields<double>(g) : mask_fields<float>(g));
    if (cudaError_t e = cell_list(g, vf::kBitNearSolid, g->near_list, &g->n_near)) return fail_cuda(g, e, "near-solid list");
    VF_CK(vf::mask_count_solid(g->mask, g->N, g->solid_count, g->stream));
    unsigned long long solids = 0;
    VF_CK(cudaMemcpyAsync(&solids, g->solid_count, sizeof(solids), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    g->has_solid = solids > 0;
    VF_CK(vf::build_stencil_mask(g->mask, g->smask, g->d.nx, g->d.ny, g->d.nz, g->stream));
    VF_CK(budget_cells(g));
    VF_CK(cudaStreamSynchronize(g->stream));
    g->mask_set = true;
    g->sigma_stale = true;   // the fields were re-masked
    drop_graphs(g);
    return VF_OK;
}

int vf_set_inflow(vf_grid* g, const uint8_t* S, const double u_set[3], double c_set, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!u_set || (mem != VF_HOST && mem != VF_DEVICE)) return set_err(g, VF_EINVAL, "vf_set_inflow: bad argument");
    if (S) {
        const void* src = stage_input(g, S, g->N, mem, &rc);
        if (rc) return rc;
        VF_CK(vf::mask_merge(g->mask, (const uint8_t*)src, vf::kBitS, g->N, g->stream));
        VF_CK(vf::build_stencil_mask(g->mask, g->smask, g->d.nx, g->d.ny, g->d.nz, g->stream));
        VF_CK(budget_cells(g));
        VF_CK(cudaStreamSynchronize(g->stream));
    }
    for (int j = 0; j < 3; ++j) g->uset[j] = u_set[j];
    g->cset = c_set;
    if (S) g->smooth_s = false;
    g->has_target = false;
    drop_graphs(g);
    return VF_OK;
}

int vf_set_inflow_tanh(vf_grid* g, const double center[3], const double width[3], const double sharpness[3],
                       const double u_set[3], double c_set)
{
    int rc = check(g);
    if (rc) return rc;
    if (!center || !width || !sharpness || !u_set) return set_err(g, VF_EINVAL, "vf_set_inflow_tanh: null argument");
    vf::TanhWindow w{};
    const double L[3] = {g->d.lx, g->d.ly, g->d.lz};
    const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
    for (int j = 0; j < 3; ++j) {
        if (!(width[j] > 0.0) || !(sharpness[j] > 0.0) || !std::isfinite(center[j]) || !std::isfinite(width[j]) ||
            !std::isfinite(sharpness[j]))
            return set_err(g, VF_EINVAL, "vf_set_inflow_tanh: width and sharpness must be positive and finite");
        w.c[j] = center[j];
        w.hw[j] = 0.5 * width[j];
        w.B[j] = sharpness[j];
        w.h[j] = L[j] / n[j];
        w.L[j] = L[j];
    }
    if (g->fp64) VF_CK(Kernels<double>::tanh_source((double*)g->sval, g->mask, w, n[0], n[1], n[2], g->stream));
    else VF_CK(Kernels<float>::tanh_source((float*)g->sval, g->mask, w, n[0], n[1], n[2], g->stream));
    VF_CK(vf::build_stencil_mask(g->mask, g->smask, n[0], n[1], n[2], g->stream));
    VF_CK(budget_cells(g));
    VF_CK(cudaStreamSynchronize(g->stream));
    for (int j = 0; j < 3; ++j) g->uset[j] = u_set[j];
    g->cset = c_set;
    g->smooth_s = true;
    g->has_target = false;
    drop_graphs(g);
    return VF_OK;
}

int vf_set_inflow_values(vf_grid* g, const void* S, int is_fp64, const double u_set[3], double c_set, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!S || !u_set || (mem != VF_HOST && mem != VF_DEVICE))
        return set_err(g, VF_EINVAL, "vf_set_inflow_values: bad argument");
    const void* src = stage_input(g, S, g->N * (is_fp64 ? 8 : 4), mem, &rc);
    if (rc) return rc;
    if (g->fp64) {
        VF_CK(Kernels<double>::convert_in(src, is_fp64, g->sval, -1, g->N, 1.0, nullptr, g->stream));
        VF_CK(Kernels<double>::source_bits(g->mask, (const double*)g->sval, g->N, g->stream));
    } else {
        VF_CK(Kernels<float>::convert_in(src, is_fp64, g->sval, -1, g->N, 1.0, nullptr, g->stream));
        VF_CK(Kernels<float>::source_bits(g->mask, (const float*)g->sval, g->N, g->stream));
    }
    VF_CK(vf::build_stencil_mask(g->mask, g->smask, g->d.nx, g->d.ny, g->d.nz, g->stream));
    VF_CK(budget_cells(g));
    VF_CK(cudaStreamSynchronize(g->stream));
    for (int j = 0; j < 3; ++j) g->uset[j] = u_set[j];
    g->cset = c_set;
    g->smooth_s = true;
    g->has_target = false;
    drop_graphs(g);
    return VF_OK;
}

int vf_set_inflow_field(vf_grid* g, const void* S, const void* targets, int is_fp64, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!S || !targets || (mem != VF_HOST && mem != VF_DEVICE))
        return set_err(g, VF_EINVAL, "vf_set_inflow_field: bad argument");
    if (!g->target && !(g->target = galloc(g, 4 * g->N * g->esz)))
        return set_err(g, VF_ENOMEM, "vf_set_inflow_field: allocation failed");
    const size_t esz_in = is_fp64 ? 8 : 4, bytes = g->N * esz_in;
    const void* src = stage_input(g, S, bytes, mem, &rc);
    if (rc) return rc;
    if (g->fp64) {
        VF_CK(Kernels<double>::convert_in(src, is_fp64, g->sval, -1, g->N, 1.0, nullptr, g->stream));
        VF_CK(Kernels<double>::source_bits(g->mask, (const double*)g->sval, g->N, g->stream));
    } else {
        VF_CK(Kernels<float>::convert_in(src, is_fp64, g->sval, -1, g->N, 1.0, nullptr, g->stream));
        VF_CK(Kernels<float>::source_bits(g->mask, (const float*)g->sval, g->N, g->stream));
    }
    VF_CK(vf::build_stencil_mask(g->mask, g->smask, g->d.nx, g->d.ny, g->d.nz, g->stream));
    VF_CK(budget_cells(g));
    for (int comp = 0; comp < 4; ++comp) {
        // one component at a time through the staging buffer (N values)
        VF_CK(cudaStreamSynchronize(g->stream));
        const void* tsrc = stage_input(g, (const char*)targets + comp * bytes, bytes, mem, &rc);
        if (rc) return rc;
        if (g->fp64) VF_CK(Kernels<double>::convert_in(tsrc, is_fp64, g->target, comp, g->N, 1.0, nullptr, g->stream));
        else VF_CK(Kernels<float>::convert_in(tsrc, is_fp64, g->target, comp, g->N, 1.0, nullptr, g->stream));
    }
    VF_CK(cudaStreamSynchronize(g->stream));
    g->smooth_s = true;
    g->has_target = true;
    drop_graphs(g);
    return VF_OK;
}

int vf_set_force_region(vf_grid* g, const uint8_t* region, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!region || (mem != VF_HOST && mem != VF_DEVICE)) return set_err(g, VF_EINVAL, "vf_set_force_region: bad argument");
    const void* src = stage_input(g, region, g->N, mem, &rc);
    if (rc) return rc;
    VF_CK(vf::mask_merge(g->mask, (const uint8_t*)src, vf::kBitForce, g->N, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_region_force(vf_grid* g, double force[3])
{
    int rc = check(g);
    if (rc) return rc;
    if (!force) return set_err(g, VF_EINVAL, "vf_region_force: null output");
    const double dV = (g->d.lx / g->d.nx) * (g->d.ly / g->d.ny) * (g->d.lz / g->d.nz);
    VF_CK(cudaMemsetAsync(g->force_acc, 0, 3 * sizeof(double), g->stream));
    if (g->fp64)
        VF_CK(vf::region_force<double>(g->q, (const double*)g->p, g->mask, g->smooth_s ? (const double*)g->sval : nullptr,
                                       g->has_target ? g->target : nullptr, flow_consts<double>(g), dV, g->force_acc,
                                       g->stream));
    else
        VF_CK(vf::region_force<float>(g->q, (const float*)g->p, g->mask, g->smooth_s ? (const float*)g->sval : nullptr,
                                      g->has_target ? g->target : nullptr, flow_consts<float>(g), dV, g->force_acc,
                                      g->stream));
    VF_CK(cudaMemcpyAsync(force, g->force_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_set_region(vf_grid* g, const uint8_t* room, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!room || (mem != VF_HOST && mem != VF_DEVICE)) return set_err(g, VF_EINVAL, "vf_set_region: bad argument");
    const void* src = stage_input(g, room, g->N, mem, &rc);
    if (rc) return rc;
    VF_CK(vf::mask_merge(g->mask, (const uint8_t*)src, vf::kBitRoom, g->N, g->stream));
    VF_CK(budget_cells(g));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_set_field(vf_grid* g, int field, const void* src, int is_fp64, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!src || field < VF_U || field > VF_P || (mem != VF_HOST && mem != VF_DEVICE))
        return set_err(g, VF_EINVAL, "vf_set_field: bad argument");
    const size_t bytes = g->N * (is_fp64 ? 8 : 4);
    const void* dsrc = stage_input(g, src, bytes, mem, &rc);
    if (rc) return rc;
    void* dst = field == VF_P ? g->p : g->q;
    const int comp = field == VF_P ? -1 : field;
    const uint8_t* mask = field == VF_P ? nullptr : g->mask;
    if (g->fp64) VF_CK(Kernels<double>::convert_in(dsrc, is_fp64, dst, comp, g->N, 1.0, mask, g->stream));
    else VF_CK(Kernels<float>::convert_in(dsrc, is_fp64, dst, comp, g->N, 1.0, mask, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    if (field <= VF_W) g->sigma_stale = true;
    return VF_OK;
}

int vf_set_time(vf_grid* g, double t, int64_t step)
{
    int rc = check(g);
    if (rc) return rc;
    if (step < 0) return set_err(g, VF_EINVAL, "vf_set_time: negative step");
    VF_CK(cudaStreamSynchronize(g->stream));
    g->step = step;
    g->t0 = t - (double)step * g->d.dt;
    long long s = step;
    VF_CK(cudaMemcpyAsync(g->dev_counters + 1, &s, sizeof(s), cudaMemcpyHostToDevice, g->stream));
    VF_CK(cudaMemcpyAsync(&g->dtctl->t_end, &t, sizeof(double), cudaMemcpyHostToDevice, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    drop_graphs(g);   // t0 is baked into the reduction launch
    return VF_OK;
}

int vf_step(vf_grid* g, int64_t n, int32_t reduce_every)
{
    int rc = check(g);
    if (rc) return rc;
    if (n < 0 || reduce_every < 0) return set_err(g, VF_EINVAL, "vf_step: negative count");
    if (!g->mask_set) return set_err(g, VF_ESTATE, "vf_step: call vf_set_mask first");
    if (g->use_graph && !g->graph_ok) {
        rc = capture_graphs(g);
        if (rc) return rc;
    }
    if (n > 0) VF_CK(vf_engine::refresh_sigma(g, g->stream));
    // with graphs and a fixed time step a recorded step's reduction runs alongside the next step's stages 1-2;
    // the last pending one is launched before returning, so the records are the same as with no lag
    const bool lag = g->use_graph && !g->dynamic;
    bool pending = false;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t s = g->step + 1;
        const bool red = reduce_every > 0 && (s % reduce_every) == 0;
        if (g->use_graph) VF_CK(cudaGraphLaunch(g->gexec[(red ? 1 : 0) | (lag && pending ? 2 : 0)], g->stream));
        else VF_CK(enqueue_step(g, g->stream, red));
        pending = lag && red;
        g->step = s;
    }
    if (pending) VF_CK(enqueue_reduction(g, g->stream));
    return VF_OK;
}

int vf_sync(vf_grid* g)
{
    int rc = check(g);
    if (rc) return rc;
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_read_field(vf_grid* g, int field, void* dst, int as_fp64, int mem)
{
    int rc = check(g);
    if (rc) return rc;
    if (!dst || field < VF_U || field > VF_P || (mem != VF_HOST && mem != VF_DEVICE))
        return set_err(g, VF_EINVAL, "vf_read_field: bad argument");
    const void* src = field == VF_P ? g->p : g->q;
    const int comp = field == VF_P ? -1 : field;
    void* out = mem == VF_DEVICE ? dst : g->staging;
    if (g->fp64) VF_CK(Kernels<double>::convert_out(src, comp, out, as_fp64, g->N, 1.0, g->stream));
    else VF_CK(Kernels<float>::convert_out(src, comp, out, as_fp64, g->N, 1.0, g->stream));
    if (mem == VF_HOST)
        VF_CK(cudaMemcpyAsync(dst, g->staging, g->N * (as_fp64 ? 8 : 4), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_reductions(vf_grid* g, vf_reduce* out)
{
    int rc = check(g);
    if (rc) return rc;
    if (!out) return set_err(g, VF_EINVAL, "vf_reductions: null output");
    const vf::ReduceArgsDev r = reduce_args(g);
    if (g->fp64) VF_CK(Kernels<double>::reduce(g->q, g->mask, flow_consts<double>(g), r, 0, g->stream));
    else VF_CK(Kernels<float>::reduce(g->q, g->mask, flow_consts<float>(g), r, 0, g->stream));
    int bad = 0;
    VF_CK(cudaMemcpyAsync(out, g->red_out, sizeof(vf_reduce), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaMemcpyAsync(&bad, g->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    if (bad) {
        VF_CK(cudaMemsetAsync(g->nonfinite, 0, sizeof(int), g->stream));
        VF_CK(cudaStreamSynchronize(g->stream));
        return set_err(g, VF_ENONFINITE, "vf_reductions: a field holds NaN or Inf");
    }
    return VF_OK;
}

int vf_history(vf_grid* g, vf_reduce* out, int64_t max_records, int64_t* count)
{
    int rc = check(g);
    if (rc) return rc;
    if (!count || (max_records > 0 && !out) || max_records < 0) return set_err(g, VF_EINVAL, "vf_history: bad argument");
    long long total = 0;
    VF_CK(cudaMemcpyAsync(&total, g->dev_counters, sizeof(total), cudaMemcpyDeviceToHost, g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    const long long cap = g->d.history_capacity;
    const long long n = std::min<long long>(std::min<long long>(total, cap), max_records);
    const long long first = total - n;
    long long done = 0;
    while (done < n) {
        const long long slot = (first + done) % cap;
        const long long run = std::min(n - done, cap - slot);
        VF_CK(cudaMemcpyAsync(out + done, g->history + slot, run * sizeof(vf_reduce), cudaMemcpyDeviceToHost,
                              g->stream));
        done += run;
    }
    VF_CK(cudaStreamSynchronize(g->stream));
    *count = n;
    return VF_OK;
}

int vf_clear_history(vf_grid* g)
{
    int rc = check(g);
    if (rc) return rc;
    VF_CK(cudaMemsetAsync(g->dev_counters, 0, sizeof(long long), g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    return VF_OK;
}

int vf_info(const vf_grid* g, double* t, int64_t* step, int64_t* cells, int64_t* device_bytes)
{
    if (!g) return VF_EINVAL;
    if (t) {
        if (g->dynamic) {
            double te = 0.0;
            if (cudaMemcpyAsync(&te, &g->dtctl->t_end, sizeof(double), cudaMemcpyDeviceToHost, g->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(g->stream) != cudaSuccess)
                return VF_ECUDA;
            *t = te;
        } else {
            *t = g->t0 + (double)g->step * g->d.dt;
        }
    }
    if (step) *step = g->step;
    if (cells) *cells = (int64_t)g->N;
    if (device_bytes) *device_bytes = (int64_t)g->bytes;
    return VF_OK;
}

int vf_particles_set(vf_grid* g, int64_t n, const double* pos, const double* vel, const double* size, double rho_p,
                     double rho_f, const double gravity[3])
{
    int rc = check(g);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!pos || !vel || !size || !gravity)) || !(rho_p > 0.0) || !(rho_f > 0.0))
        return set_err(g, VF_EINVAL, "vf_particles_set: bad argument");
    const double L[3] = {g->d.lx, g->d.ly, g->d.lz};
    for (int64_t i = 0; i < n; ++i) {
        if (!(size[i] > 0.0)) return set_err(g, VF_EINVAL, "vf_particles_set: sizes must be positive");
        for (int k = 0; k < 3; ++k)
            if (!(pos[3 * i + k] >= 0.0 && pos[3 * i + k] < L[k]) || !std::isfinite(vel[3 * i + k]))
                return set_err(g, VF_EINVAL, "vf_particles_set: positions must lie in the box");
    }
    VF_CK(cudaStreamSynchronize(g->stream));
    free_particles(g);
    drop_graphs(g);
    if (n == 0) return VF_OK;
    // one buffer: x, y, z, u, v, w, d (n doubles each), then the states (n ints)
    const size_t bytes = ((size_t)n * 7 * sizeof(double) + (size_t)n * sizeof(int) + 255) & ~(size_t)255;
    void* buf = nullptr;
    if (g->have_alloc) buf = g->alloc.alloc(bytes, (void*)g->stream, g->alloc.ctx);
    else if (cudaMallocAsync(&buf, bytes, g->stream) != cudaSuccess) { cudaGetLastError(); buf = nullptr; }
    if (!buf) return set_err(g, VF_ENOMEM, "vf_particles_set: allocation failed");
    g->particle_buf = buf;
    g->particle_bytes = bytes;
    g->bytes += bytes;
    std::vector<double> host((size_t)n * 7);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            host[(size_t)k * n + i] = pos[3 * i + k];
            host[(size_t)(3 + k) * n + i] = vel[3 * i + k];
        }
    for (int64_t i = 0; i < n; ++i) host[(size_t)6 * n + i] = size[i];
    double* dbuf = (double*)buf;
    VF_CK(cudaMemcpyAsync(dbuf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    int* state = (int*)(dbuf + (size_t)n * 7);
    VF_CK(cudaMemsetAsync(state, 0, (size_t)n * sizeof(int), g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));   // host staging dies here
    vf::ParticleArgs& P = g->particles;
    P = vf::ParticleArgs{};
    P.n = n;
    for (int k = 0; k < 3; ++k) {
        P.pos[k] = dbuf + (size_t)k * n;
        P.vel[k] = dbuf + (size_t)(3 + k) * n;
        P.h[k] = L[k] / (k == 0 ? g->d.nx : k == 1 ? g->d.ny : g->d.nz);
        P.ih[k] = 1.0 / P.h[k];
        P.L[k] = L[k];
        P.g[k] = gravity[k];
    }
    P.size = dbuf + (size_t)6 * n;
    P.state = state;
    P.nx = g->d.nx; P.ny = g->d.ny; P.nz = g->d.nz;
    P.nu = g->d.nu;
    P.rho_p = rho_p;
    P.rho_f = rho_f;
    P.dt = g->d.dt;
    return VF_OK;
}

int vf_particles_read(vf_grid* g, double* pos, double* vel, int32_t* deposited)
{
    int rc = check(g);
    if (rc) return rc;
    const int64_t n = g->particles.n;
    if (n == 0) return VF_OK;
    std::vector<double> host((size_t)n * 6);
    std::vector<int> st((size_t)n);
    VF_CK(cudaMemcpyAsync(host.data(), g->particles.pos[0], host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          g->stream));
    VF_CK(cudaMemcpyAsync(st.data(), g->particles.state, st.size() * sizeof(int), cudaMemcpyDeviceToHost,
                          g->stream));
    VF_CK(cudaStreamSynchronize(g->stream));
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            if (pos) pos[3 * i + k] = host[(size_t)k * n + i];
            if (vel) vel[3 * i + k] = host[(size_t)(3 + k) * n + i];
        }
    if (deposited)
        for (int64_t i = 0; i < n; ++i) deposited[i] = st[(size_t)i];
    return VF_OK;
}

int vf_particles_count(const vf_grid* g, int64_t* n)
{
    if (!g || !n) return VF_EINVAL;
    *n = g->particles.n;
    return VF_OK;
}

int vf_poisson_solve(vf_grid* g, const void* f, void* p)
{
    int rc = check(g);
    if (rc) return rc;
    if (!f || !p) return set_err(g, VF_EINVAL, "vf_poisson_solve: null pointer");
    if (g->fp64) {
        const PoissonArgs<double> a = poisson_args<double>(g, (double*)f, (double*)p, 0);
        VF_CK(Kernels<double>::poisson_iteration(a, 1, g->stream));
    } else {
        const PoissonArgs<float> a = poisson_args<float>(g, (float*)f, (float*)p, 0);
        VF_CK(Kernels<float>::poisson_iteration(a, 1, g->stream));
    }
    return VF_OK;
}

int vf_profile_steps(vf_grid* g, int64_t n, int32_t reduce_every, double* phase_ms, int64_t* launches)
{
    int rc = check(g);
    if (rc) return rc;
    if (n < 0 || reduce_every < 0 || !phase_ms || !launches) return set_err(g, VF_EINVAL, "vf_profile_steps: bad argument");
    if (!g->mask_set) return set_err(g, VF_ESTATE, "vf_profile_steps: call vf_set_mask first");
    if (n > 0) VF_CK(vf_engine::refresh_sigma(g, g->stream));
    for (int64_t i = 0; i < n; ++i) {
        PhaseRecorder rec;
        rec.stream = g->stream;
        cudaEvent_t start;
        VF_CK(cudaEventCreate(&start));
        VF_CK(cudaEventRecord(start, g->stream));
        const vf::LaunchHook hook{&PhaseRecorder::hook, &rec};
        const int64_t s = g->step + 1;
        const bool red = reduce_every > 0 && (s % reduce_every) == 0;
        cudaError_t e = enqueue_step(g, g->stream, red, &hook);
        g->step = s;
        if (e == cudaSuccess) e = rec.err;
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        cudaEvent_t prev = start;
        for (size_t k = 0; e == cudaSuccess && k < rec.events.size(); ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, prev, rec.events[k]);
            const int ph = rec.phases[k];
            if (e == cudaSuccess && ph >= 0 && ph < VF_N_PHASES) {
                phase_ms[ph] += ms;
                launches[ph] += 1;
            }
            prev = rec.events[k];
        }
        cudaEventDestroy(start);
        for (cudaEvent_t ev : rec.events) cudaEventDestroy(ev);
        if (e != cudaSuccess) return fail_cuda(g, e, "vf_profile_steps");
    }
    return VF_OK;
}

const char* vf_phase_name(int phase)
{
    static const char* names[VF_N_PHASES] = {"stage1", "stage2", "stage3", "stage4", "div", "fft_x_fwd",
                                             "fft_y_fwd", "fft_z_solve", "fft_y_inv", "fft_x_inv", "project",
                                             "filter", "reduce", "poisson_rhs", "fft_yz_solve", "adjust_dt",
                                             "particles"};
    if (phase < 0 || phase >= VF_N_PHASES) return "unknown";
    return names[phase];
}

int vf_abi_sizes(int64_t out[4])
{
    if (!out) return VF_EINVAL;
    out[0] = (int64_t)sizeof(vf_grid_desc);
    out[1] = (int64_t)sizeof(vf_reduce);
    out[2] = (int64_t)sizeof(vf_batch_desc);
    out[3] = (int64_t)sizeof(vf_tiles);
    return VF_OK;
}

const char* vf_status_string(int status)
{
    if (status > 0 || status < VF_ETIMEOUT) return "VF_UNKNOWN";
    return kStatusNames[-status];
}

const char* vf_last_error(const vf_grid* g)
{
    if (!g) return "null grid";
    return g->err.c_str();
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------------------
// Launch tiles and the autotuner
// ------------------------------------------------------------------------------------------------------------
namespace {

struct TileKey {
    int nx, ny, nz, precision;
    bool operator<(const TileKey& o) const
    {
        if (nx != o.nx) return nx < o.nx;
        if (ny != o.ny) return ny < o.ny;
        if (nz != o.nz) return nz < o.nz;
        return precision < o.precision;
    }
};

std::mutex& tile_mutex()
{
    static std::mutex m;
    return m;
}

std::map<TileKey, vf_tiles>& tile_cache()
{
    static std::map<TileKey, vf_tiles> c;
    return c;
}

bool tiles_valid(const vf_tiles& t)
{
    for (int v : {t.zc_stage, t.zc_div, t.zc_project, t.zc_filter})
        if (v < vf::kZChunkMin || v > vf::kZChunkMax) return false;
    return true;
}

// Mean milliseconds of `reps` enqueues of `launch` on the grid's stream, after one warm-up enqueue.
template <typename F>
cudaError_t time_launches(cudaStream_t st, int reps, F&& launch, float* ms)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e == cudaSuccess) *ms /= (float)reps;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

// Each family is timed on the grid's arrays exactly as a step launches it, except that every output goes to a
// scratch array: stage states (qa, qb, acc), divergence (f), projection (qb, no step tick), filter (acc, with its
// divergence records, read only by a reduction launched after it); with the filter off the standalone reduction,
// its record and non-finite flag redirected into the staging buffer, no history.
template <typename T>
int autotune_t(vf_grid* g, int reps, vf_tiles* best)
{
    static const int kCand[] = {4, 8, 16, 32};
    FlowConsts<T> k = flow_consts<T>(g);
    const cudaStream_t st = g->stream;
    vf::ReduceArgsDev ra = reduce_args(g);
    const bool redirect = g->N * 8 >= sizeof(vf_reduce) + 256;
    if (redirect) {
        ra.out = (vf_reduce*)g->staging;
        ra.nonfinite = (int*)((char*)g->staging + ((sizeof(vf_reduce) + 255) & ~(size_t)255));
    }
    int chosen[vf::kZcKinds];
    for (int fam = 0; fam < vf::kZcKinds; ++fam) {
        float best_ms = 0.f;
        chosen[fam] = g->zc[fam];
        int prev = 0;
        for (int c : kCand) {
            // chunks at or beyond nz all launch one CTA per column: time only the first of them
            const int eff = std::min(c, k.nz);
            if (eff == prev) continue;
            prev = eff;
            k.zc[fam] = c;
            auto launch = [&]() -> cudaError_t {
                StageArgs<T> a{};
                a.mask = g->mask;
                a.smask = g->smask;
                a.qn = g->q;
                cudaError_t e = cudaSuccess;
                switch (fam) {
                    case vf::kZcStage:
                        a.qs = g->q; a.out = g->qa;
                        if ((e = Kernels<T>::stage(1, a, k, st)) != cudaSuccess) return e;
                        a.qs = g->qa; a.out = g->qb;
                        if ((e = Kernels<T>::stage(2, a, k, st)) != cudaSuccess) return e;
                        a.qs = g->qb; a.out = g->acc;
                        if ((e = Kernels<T>::stage(3, a, k, st)) != cudaSuccess) return e;
                        a.qs = g->acc; a.q2 = g->qa; a.q3 = g->qb; a.out = g->qa;
                        return Kernels<T>::stage(4, a, k, st);
                    case vf::kZcDiv: return Kernels<T>::divergence(g->qa, (T*)g->f, k, st);
                    case vf::kZcProject:
                        return Kernels<T>::project(g->qa, (const T*)g->p, g->qb, g->mask, nullptr, k, st);
                    default:
                        if (!g->d.filter) return Kernels<T>::reduce(g->qb, g->mask, k, ra, 0, st);
                        return Kernels<T>::filter(g->qb, g->acc, g->mask, k, &ra, st);   // scratch records only
                }
            };
            float ms = 0.f;
            const cudaError_t e = time_launches(st, reps, launch, &ms);
            if (e != cudaSuccess) return fail_cuda(g, e, "vf_autotune");
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                chosen[fam] = c;
            }
        }
        k.zc[fam] = chosen[fam];
    }
    best->zc_stage = chosen[0];
    best->zc_div = chosen[1];
    best->zc_project = chosen[2];
    best->zc_filter = chosen[3];
    // FFT radix schedules (generic passes only): each axis in turn, the others at their best so far, timed as one
    // Poisson solve of the scratch array qa into qb (no Eq. 9 correction)
    int sched[3] = {g->fft_sched[0], g->fft_sched[1], g->fft_sched[2]};
    if (!g->reg) {
        int len[3];
        fft_lengths(g, len);
        for (int axis = 0; axis < 3; ++axis) {
            const int nc = (int)vf::fft_schedules(len[axis]).size();
            float best_ms = 0.f;
            int pick = sched[axis];
            for (int c = 0; c < nc; ++c) {
                int trial[3] = {sched[0], sched[1], sched[2]};
                trial[axis] = c;
                int rc = set_fft_sched(g, trial);
                if (rc) return rc;
                const PoissonArgs<T> pa = poisson_args<T>(g, (T*)g->qa, (T*)g->qb, 0);
                auto launch = [&]() -> cudaError_t { return Kernels<T>::poisson_iteration(pa, 1, st); };
                float ms = 0.f;
                const cudaError_t e = time_launches(st, reps, launch, &ms);
                if (e != cudaSuccess) return fail_cuda(g, e, "vf_autotune");
                if (best_ms == 0.f || ms < best_ms) {
                    best_ms = ms;
                    pick = c;
                }
            }
            sched[axis] = pick;
        }
        const int rc = set_fft_sched(g, sched);
        if (rc) return rc;
    }
    best->fft_x = sched[0];
    best->fft_y = sched[1];
    best->fft_z = sched[2];
    return VF_OK;
}

int apply_tiles(vf_grid* g, const vf_tiles& t)
{
    g->zc[vf::kZcStage] = t.zc_stage;
    g->zc[vf::kZcDiv] = t.zc_div;
    g->zc[vf::kZcProject] = t.zc_project;
    g->zc[vf::kZcFilter] = t.zc_filter;
    drop_graphs(g);
    const int idx[3] = {t.fft_x, t.fft_y, t.fft_z};
    if (idx[0] == g->fft_sched[0] && idx[1] == g->fft_sched[1] && idx[2] == g->fft_sched[2]) return VF_OK;
    return set_fft_sched(g, idx);
}

}  // namespace

extern "C" {

int vf_get_tiles(const vf_grid* g, vf_tiles* out)
{
    if (!g || !out) return VF_EINVAL;
    out->zc_stage = g->zc[vf::kZcStage];
    out->zc_div = g->zc[vf::kZcDiv];
    out->zc_project = g->zc[vf::kZcProject];
    out->zc_filter = g->zc[vf::kZcFilter];
    out->fft_x = g->fft_sched[0];
    out->fft_y = g->fft_sched[1];
    out->fft_z = g->fft_sched[2];
    return VF_OK;
}

int vf_fft_path(const vf_grid* g, int32_t* path)
{
    if (!g || !path) return VF_EINVAL;
    *path = !g->reg ? VF_FFT_GENERIC : (g->reg_tile ? VF_FFT_REGISTER_TILE : VF_FFT_REGISTER_PLANE);
    return VF_OK;
}

int vf_set_tiles(vf_grid* g, const vf_tiles* t)
{
    int rc = check(g);
    if (rc) return rc;
    if (!t || !tiles_valid(*t)) return set_err(g, VF_EINVAL, "vf_set_tiles: chunk out of range");
    const int idx[3] = {t->fft_x, t->fft_y, t->fft_z};
    if (!fft_indices_valid(g, idx)) return set_err(g, VF_EINVAL, "vf_set_tiles: FFT schedule index out of range");
    VF_CK(cudaStreamSynchronize(g->stream));
    return apply_tiles(g, *t);
}

int vf_fft_schedules(int32_t n, int32_t index, int32_t* radices, int32_t max_radices)
{
    if (!radices || index < 0 || max_radices < 1) return VF_EINVAL;
    const std::vector<std::vector<int>> c = vf::fft_schedules(n);
    if (index >= (int)c.size()) return 0;
    const std::vector<int>& r = c[index];
    if ((int)r.size() > max_radices) return VF_EINVAL;
    for (size_t i = 0; i < r.size(); ++i) radices[i] = r[i];
    return (int)r.size();
}

int vf_autotune(vf_grid* g, int32_t reps, vf_tiles* chosen)
{
    int rc = check(g);
    if (rc) return rc;
    if (reps < 1 || reps > 1000) return set_err(g, VF_EINVAL, "vf_autotune: reps outside [1, 1000]");
    VF_CK(cudaStreamSynchronize(g->stream));
    vf_tiles t{};
    rc = g->fp64 ? autotune_t<double>(g, reps, &t) : autotune_t<float>(g, reps, &t);
    if (rc) return rc;
    VF_CK(cudaStreamSynchronize(g->stream));
    if ((rc = apply_tiles(g, t))) return rc;
    {
        std::lock_guard<std::mutex> lock(tile_mutex());
        tile_cache()[TileKey{g->d.nx, g->d.ny, g->d.nz, g->d.precision}] = t;
    }
    if (chosen) *chosen = t;
    return VF_OK;
}

int vf_tile_cache_lookup(int32_t nx, int32_t ny, int32_t nz, int32_t precision, vf_tiles* out)
{
    std::lock_guard<std::mutex> lock(tile_mutex());
    auto it = tile_cache().find(TileKey{nx, ny, nz, precision});
    if (it == tile_cache().end()) return 0;
    if (out) *out = it->second;
    return 1;
}

int vf_tile_cache_clear(void)
{
    std::lock_guard<std::mutex> lock(tile_mutex());
    tile_cache().clear();
    return VF_OK;
}

int64_t vf_tile_cache_size(void)
{
    std::lock_guard<std::mutex> lock(tile_mutex());
    return (int64_t)tile_cache().size();
}

int vf_tile_cache_entry(int64_t i, int32_t key[4], vf_tiles* out)
{
    if (!key || !out) return VF_EINVAL;
    std::lock_guard<std::mutex> lock(tile_mutex());
    if (i < 0 || i >= (int64_t)tile_cache().size()) return VF_EINVAL;
    auto it = tile_cache().begin();
    std::advance(it, (long)i);
    key[0] = it->first.nx;
    key[1] = it->first.ny;
    key[2] = it->first.nz;
    key[3] = it->first.precision;
    *out = it->second;
    return VF_OK;
}

int vf_tile_cache_insert(int32_t nx, int32_t ny, int32_t nz, int32_t precision, const vf_tiles* t)
{
    if (!t || !tiles_valid(*t) || (precision != VF_FP64 && precision != VF_FP32_MIXED)) return VF_EINVAL;
    if (!smooth235_even(nx) || !smooth235_even(ny) || !smooth235_even(nz)) return VF_ESIZE;
    if ((long long)nx * ny * nz > kMaxCells) return VF_ESIZE;
    const int len[3] = {nx / 2, ny, nz}, idx[3] = {t->fft_x, t->fft_y, t->fft_z};
    for (int a = 0; a < 3; ++a)
        if (idx[a] < 0 || idx[a] >= (int)vf::fft_schedules(len[a]).size()) return VF_EINVAL;
    std::lock_guard<std::mutex> lock(tile_mutex());
    tile_cache()[TileKey{nx, ny, nz, precision}] = *t;
    return VF_OK;
}

}  // extern "C"
