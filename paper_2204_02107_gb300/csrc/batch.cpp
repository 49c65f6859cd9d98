// Batch engine: many rooms of uneven size advanced together (declared in include/ventflow.h, vf_batch_*).
//
// A batch owns one grid per occupied slot.  One step of the batch is one CUDA graph with an independent branch per
// active room: the graph is captured by forking the batch stream into every room's capture stream, enqueuing that
// room's step (the same launches a single-room vf_step replays) and joining back.  A single graph launch therefore
// advances every room, and the rooms' kernels run concurrently on the GPU.  Each room's arithmetic is exactly the
// one it would do alone, so a room's fields are bitwise the same alone and in any mix.
//
// Launch tiles: with autotune set, the first room of each (nx, ny, nz, precision) is autotuned on admission and
// the result cached; later rooms of that shape, and grids created alone, take the cached tiles.
//
// Admission: a room is accepted only while the bytes its grid allocates (vf_grid_bytes) fit in the batch's budget.
// Rooms run for their own number of steps; vf_batch_step advances in chunks that end when some room finishes, so
// no room is stepped past its target.  Finished rooms keep their results until vf_batch_remove.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "grid.h"

struct vf_batch_slot {
    vf_grid* g = nullptr;
    int64_t remaining = 0;    // steps still to run
    int64_t target = 0;       // steps requested
    bool done = false;        // reached its target; results readable, no longer stepped
    size_t bytes = 0;
    cudaEvent_t join = nullptr;
};

struct vf_batch {
    vf_batch_desc d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t fork = nullptr;
    std::vector<vf_batch_slot> slots;
    size_t bytes_in_use = 0;
    int64_t batch_step = 0;
    cudaGraphExec_t exec[2]{nullptr, nullptr};
    bool graph_ok = false;
    std::string err;
    int status = VF_OK;
};

namespace {

int bfail(vf_batch* b, cudaError_t e, const char* what)
{
    b->status = VF_ECUDA;
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return VF_ECUDA;
}

#define VB_CK(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return bfail(b, e_, #call);           \
    } while (0)

void drop_graphs(vf_batch* b)
{
    for (int i = 0; i < 2; ++i)
        if (b->exec[i]) { cudaGraphExecDestroy(b->exec[i]); b->exec[i] = nullptr; }
    b->graph_ok = false;
}

bool stepping(const vf_batch_slot& s) { return s.g && !s.done && s.remaining > 0; }

long long cells_of(const vf_grid* g) { return (long long)g->d.nx * g->d.ny * g->d.nz; }

// Rooms run in lanes: chains of rooms, each room's step after the previous room's of its lane.  As many lanes as
// keep the Poisson working set of the rooms in flight (right-hand side, spectrum and pressure: 3 values a cell)
// within 60 % of L2, so that each room's four solves find their spectrum still in L2, but at least 8, which keep
// the SMs busy between the launches of a room; all rooms in parallel left the spectra of 64 rooms competing for
// L2 (mixed 64-room batch on GB300: 8.0 Gcell/s with every room a branch, 8.3 / 8.7 / 8.8 / 8.7 / 8.6 / 8.3 with
// 4 / 6 / 8 / 10 / 16 / 32 lanes; 64 rooms of 128 x 64 x 64: 9.1 all parallel, 9.4 with 12 lanes; 8 rooms of
// 256 x 128 x 128: 11.1 all parallel, 10.9 with 2 lanes).  VF_BATCH_LANES overrides the count (0: every room its
// own branch).
int lane_count(const std::vector<vf_batch_slot*>& rooms)
{
    if (rooms.empty()) return 0;
    if (const char* lv = std::getenv("VF_BATCH_LANES")) return std::max(0, std::atoi(lv));
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        l2 <= 0)
        return 0;
    double per_room = 0.0;
    for (const vf_batch_slot* s : rooms)
        per_room += (double)cells_of(s->g) * 3.0 * (s->g->d.precision == VF_FP32_MIXED ? 4.0 : 8.0);
    per_room /= (double)rooms.size();
    const int lanes = (int)(0.6 * l2 / per_room);
    return std::min(std::max(8, lanes), (int)rooms.size());
}

// One graph per reduction variant: fork the batch stream into the lanes, enqueue each room's step on its capture
// stream after the previous room of its lane (longest rooms first, each to the least loaded lane), join back.
int capture(vf_batch* b)
{
    drop_graphs(b);
    for (int v = 0; v < 2; ++v) {
        cudaGraph_t graph = nullptr;
        VB_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        cudaError_t e = cudaEventRecord(b->fork, b->stream);
        std::vector<vf_batch_slot*> order;
        for (vf_batch_slot& s : b->slots)
            if (stepping(s)) order.push_back(&s);
        const int lanes = lane_count(order);
        std::vector<cudaEvent_t> tail;
        std::vector<long long> load;
        if (lanes > 0) {
            std::stable_sort(order.begin(), order.end(), [](const vf_batch_slot* a, const vf_batch_slot* c) {
                return cells_of(a->g) > cells_of(c->g); });
            tail.assign((size_t)lanes, b->fork);
            load.assign((size_t)lanes, 0);
        }
        for (vf_batch_slot* sp : order) {
            vf_batch_slot& s = *sp;
            if (e != cudaSuccess) break;
            int l = -1;
            if (lanes > 0) {
                l = 0;
                for (int i = 1; i < lanes; ++i) if (load[i] < load[l]) l = i;
                load[l] += cells_of(s.g);
            }
            e = cudaStreamWaitEvent(s.g->cap_stream, l < 0 ? b->fork : tail[l], 0);
            if (e == cudaSuccess) e = vf_engine::enqueue_step(s.g, s.g->cap_stream, v == 1);
            if (e == cudaSuccess) e = cudaEventRecord(s.join, s.g->cap_stream);
            if (l >= 0) tail[l] = s.join;
            else if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, s.join, 0);
        }
        for (cudaEvent_t t : tail)
            if (e == cudaSuccess && t != b->fork) e = cudaStreamWaitEvent(b->stream, t, 0);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return bfail(b, e, "batch capture"); }
        if (e2 != cudaSuccess) return bfail(b, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec[v], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, e, "cudaGraphInstantiate");
    }
    b->graph_ok = true;
    return VF_OK;
}

}  // namespace

extern "C" {

int vf_batch_create(const vf_batch_desc* d, vf_batch** out)
{
    if (!d || !out || d->max_slots < 1 || d->hbm_budget_bytes <= 0 || d->reduce_every < 0 || d->autotune < 0 ||
        d->autotune > 1000)
        return VF_EINVAL;
    *out = nullptr;
    vf_batch* b = new vf_batch();
    b->d = *d;
    if (d->cuda_stream) {
        b->stream = (cudaStream_t)d->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return VF_ECUDA; }
        b->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return VF_ECUDA;
    }
    b->slots.resize((size_t)d->max_slots);
    *out = b;
    return VF_OK;
}

int vf_batch_destroy(vf_batch* b)
{
    if (!b) return VF_OK;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (vf_batch_slot& s : b->slots) {
        if (s.g) vf_destroy(s.g);
        if (s.join) cudaEventDestroy(s.join);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return VF_OK;
}

int vf_batch_add(vf_batch* b, const vf_grid_desc* gd, const uint8_t* beta, const uint8_t* S, const uint8_t* room,
                 const double u_set[3], double c_set, const void* c0, int c0_is_fp64, int64_t steps, int mem,
                 int32_t* slot)
{
    if (!b || !gd || !beta || !u_set || !slot || steps < 0 || (mem != VF_HOST && mem != VF_DEVICE)) return VF_EINVAL;
    if (b->status) return b->status;
    *slot = -1;
    int free_slot = -1;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (!b->slots[i].g) { free_slot = (int)i; break; }
    if (free_slot < 0) { b->err = "vf_batch_add: no free slot"; return VF_ENOMEM; }
    // the grid keeps its own stream for uploads and reads, so adding a room never waits for the rooms already
    // running; its steps run inside the batch graph on the batch stream
    vf_grid_desc desc = *gd;
    desc.cuda_stream = nullptr;
    const size_t need = vf_engine::grid_bytes(desc);
    if (b->bytes_in_use + need > (size_t)b->d.hbm_budget_bytes) {
        b->err = "vf_batch_add: over the memory budget";
        return VF_ENOMEM;
    }
    vf_grid* g = nullptr;
    int rc = vf_create_grid(&desc, &g);
    if (rc) { b->err = "vf_batch_add: vf_create_grid failed"; return rc; }
    auto undo = [&](int code) { vf_destroy(g); return code; };
    if ((rc = vf_set_mask(g, beta, mem))) return undo(rc);
    if ((rc = vf_set_inflow(g, S, u_set, c_set, mem))) return undo(rc);
    if (room && (rc = vf_set_region(g, room, mem))) return undo(rc);
    if (c0 && (rc = vf_set_field(g, VF_C, c0, c0_is_fp64, mem))) return undo(rc);
    if (b->d.autotune > 0 && vf_tile_cache_lookup(desc.nx, desc.ny, desc.nz, desc.precision, nullptr) == 0) {
        // a shape seen for the first time: tune on an idle GPU (the running rooms are drained first)
        const cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) { vf_destroy(g); return bfail(b, e, "vf_batch_add: drain before autotune"); }
        if ((rc = vf_autotune(g, b->d.autotune, nullptr))) return undo(rc);
    }
    vf_batch_slot& s = b->slots[(size_t)free_slot];
    if (!s.join && cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming) != cudaSuccess) return undo(VF_ECUDA);
    s.g = g;
    s.remaining = steps;
    s.target = steps;
    s.done = steps == 0;
    s.bytes = need;
    b->bytes_in_use += need;
    drop_graphs(b);
    *slot = free_slot;
    return VF_OK;
}

int vf_batch_step(vf_batch* b, int64_t n)
{
    if (!b || n < 0) return VF_EINVAL;
    if (b->status) return b->status;
    while (n > 0) {
        int64_t chunk = n;
        bool any = false;
        for (const vf_batch_slot& s : b->slots)
            if (stepping(s)) { chunk = std::min(chunk, s.remaining); any = true; }
        if (!any) break;
        if (!b->graph_ok) {
            int rc = capture(b);
            if (rc) return rc;
        }
        // rooms with a dynamic time step whose fields changed: their Courant rate, ahead of the graph
        for (vf_batch_slot& s : b->slots)
            if (stepping(s)) VB_CK(vf_engine::refresh_sigma(s.g, b->stream));
        const int re = b->d.reduce_every;
        for (int64_t i = 0; i < chunk; ++i) {
            const int64_t s = b->batch_step + 1;
            const bool red = re > 0 && (s % re) == 0;
            VB_CK(cudaGraphLaunch(b->exec[red ? 1 : 0], b->stream));
            b->batch_step = s;
        }
        bool finished = false;
        for (vf_batch_slot& s : b->slots) {
            if (!stepping(s)) continue;
            s.remaining -= chunk;
            s.g->step += chunk;
            if (s.remaining == 0) { s.done = true; finished = true; }
        }
        if (finished) drop_graphs(b);
        n -= chunk;
    }
    return VF_OK;
}

int vf_batch_sync(vf_batch* b)
{
    if (!b) return VF_EINVAL;
    VB_CK(cudaStreamSynchronize(b->stream));
    return VF_OK;
}

int vf_batch_poll(vf_batch* b, int32_t* done_slots, int32_t max_slots, int32_t* n_done)
{
    if (!b || !n_done || (max_slots > 0 && !done_slots)) return VF_EINVAL;
    VB_CK(cudaStreamSynchronize(b->stream));
    int32_t k = 0;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (b->slots[i].g && b->slots[i].done) {
            if (k < max_slots) done_slots[k] = (int32_t)i;
            ++k;
        }
    *n_done = k;
    return VF_OK;
}

vf_grid* vf_batch_grid(vf_batch* b, int32_t slot)
{
    if (!b || slot < 0 || (size_t)slot >= b->slots.size()) return nullptr;
    return b->slots[(size_t)slot].g;
}

int vf_batch_remove(vf_batch* b, int32_t slot)
{
    if (!b || slot < 0 || (size_t)slot >= b->slots.size() || !b->slots[(size_t)slot].g) return VF_EINVAL;
    VB_CK(cudaStreamSynchronize(b->stream));
    vf_batch_slot& s = b->slots[(size_t)slot];
    vf_destroy(s.g);
    s.g = nullptr;
    b->bytes_in_use -= s.bytes;
    s.bytes = 0;
    s.remaining = s.target = 0;
    s.done = false;
    drop_graphs(b);
    return VF_OK;
}

int vf_batch_info(const vf_batch* b, int32_t* active, int32_t* done, int64_t* bytes_in_use, int64_t* batch_steps)
{
    if (!b) return VF_EINVAL;
    int32_t a = 0, dn = 0;
    for (const vf_batch_slot& s : b->slots) {
        if (!s.g) continue;
        if (s.done) ++dn;
        else ++a;
    }
    if (active) *active = a;
    if (done) *done = dn;
    if (bytes_in_use) *bytes_in_use = (int64_t)b->bytes_in_use;
    if (batch_steps) *batch_steps = b->batch_step;
    return VF_OK;
}

const char* vf_batch_last_error(const vf_batch* b)
{
    if (!b) return "null batch";
    return b->err.c_str();
}

}  // extern "C"
