// pic_abi.cu -- host side of the C ABI declared in include/pic.h.
//
// Owns the device state of one or more independent runs, validates
// configurations, orders every device operation on the borrowed stream and
// replays each kind of timestep (with / without the periodic tile sort) as a
// captured CUDA graph.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <utility>
#include <new>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enums; the encoder is resolved at run time

#include "pic.h"
#include "common.cuh"
#include "internal.h"

using namespace pic;

namespace {

constexpr int kTail = 256;              // particles per tail work item (at least)
// profiling events of one step: the marks that open phases 0..PIC_PH_WINDOW in
// order, the end mark, and the start of the zero-field kernel (the end of
// PIC_PH_PUSH_ZERO is the mark that opens PIC_PH_YEE_B1)
constexpr int kMarkEnd = PIC_PH_WINDOW + 1, kMarkZero = kMarkEnd + 1, kEvPerStep = kMarkZero + 1;
constexpr int kSortMaxAdaptive = 32;    // default longest interval between sorts, adaptive policy

struct HostRun {
    pic_config cfg;
    pic_species sp;
    std::vector<double> knots;
    Run r;
    long long inject_per_shift = 0;
    long long loaded = 0;   // particles loaded (their ids are 0 .. loaded-1)
    double *rho = nullptr;  // diagnostics scratch (charge density, FP64)
    float *rho32 = nullptr; // FP32 copy for pic_read_fields(PIC_RHO)
};

// Reverse-mode state: checkpoints, one recorded segment, adjoint arrays.
struct Ckpt {
    PartCopy pc;
    float *E[3], *B[3];
    RunState *st;
    double time;
};
struct Rec {
    PartCopy pc;
    int32_t *src;       // after a sort: the slot each particle had before it
    float *E[3], *B[3];
    int32_t *tile_off;  // tile offsets of the last sort (the slots' grouping)
    RunState *st;       // the run state the push of this step starts from (device)
    double time;
    bool sorted;  // a tile sort ran just before this record (slot order changed)
};
struct Adj {
    int K = 1, total = 0, nck = 0;
    long long nid = 0;     // particle ids the adjoint arrays hold (loaded + injected during the run)
    long long nslot = 0;   // particle slots the records and slot adjoints hold
    long long nload = 0;   // loaded particles (ids 0 .. nload-1; dL/dw is reported for them)
    AdjPtrs A{};
    float *zb = nullptr;
    double *la0 = nullptr, *red = nullptr, *dk = nullptr;
    std::vector<Ckpt> ck;
    std::vector<Rec> rec;
    bool rec_on = false, save_ckpt = true, spent = false;
    int rec_base = 0;
    int keep = 0;       // the last `keep` segments are recorded by the forward run, not recomputed
    int keep_base = 0;  // first step of those segments
};

}  // namespace

struct pic_s {
    int nruns = 0, cur = 0, dim = 2, order = 2;
    cudaStream_t stream = nullptr;
    pic_alloc_fn alloc = nullptr;
    pic_free_fn free = nullptr;
    void *ctx = nullptr;
    std::vector<HostRun> runs;
    std::vector<void *> allocs;
    Run *d_runs = nullptr;
    RunState *d_states = nullptr;
    Item *d_items = nullptr;
    int n_items = 0;
    int n_tail = 0;               // leading tail items of d_items
    bool classify = true;         // stream the zero-field tiles (launch_classify)
    bool zero_wide = true;        // every run's tiles hold >= 4096 particles (streaming kernel variant)
    Item *d_live = nullptr;       // per step: tail items, then the live tiles
    Item *d_zero = nullptr;       // per step: the zero-field tiles
    Item *d_nq = nullptr;         // per step: the rows of tiles with a tile that is not quiet (field update, next J reset)
    bool field_list = false;      // the field update walks d_nq (quiet tiles on, 4-cell rows)
    int *d_cnt = nullptr;         // [4]: live tiles, zero tiles, work queue of the live kernel, spare
    int stage_lo[3] = {0, 0, 0}, stage_len[3] = {1, 1, 1};  // field region a tile stages
    int *d_seg = nullptr;  // 5 segment tables of nruns+1 ints
    int *d_scan = nullptr; // per-block sums of the sort's key scan
    Seg seg_cells{}, seg_planes{}, seg_parts{}, seg_inject{}, seg_keys{};
    int sort_sub = 1;
    bool sort_rows = true;  // each tile's particles grouped by row of cells along x
    int quiet_mode = 0;     // pic_tuning.quiet_tiles
    bool use_tma = false;
    bool split = false;  // virtual-trajectory deposit (pic_tuning.deposit = 1)
    bool j4 = false;     // four-component current nodes (pic_tuning.j_layout = 1)
    int variant() const { return use_tma ? 1 : (split ? 2 : 0); }
    bool sort_adaptive = true;  // the device decides when to sort (sort_decide_kernel)
    int adjoint_keep = 0;
    bool yee_quad = true;  // every run: rows of a multiple of 4 cells, 16-byte aligned field arrays
    size_t push_smem = 0;
    int block = 256, sort_interval = 4, fixed_interval = 4, drift = 1, tile[3] = {16, 16, 1};
    bool use_graph = true;
    bool started = false, need_sort = true, any_open = false, any_window = false;
    int since_sort = 0;
    int max_tiles = 0;
    double *d_diag = nullptr;
    unsigned long long *d_count = nullptr;
    int *d_queue = nullptr;  // work-queue counter of the persistent push kernel
    bool persistent = false;
    int num_sms = 1;
    int tail_block = 256;  // particles per tail work item (build_items)
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // [sort forced + 2 * adaptive]
    // phase profiling: events[step][kEvPerStep]
    std::vector<cudaEvent_t> prof_events;
    int prof_max = 0, prof_steps = 0;
    bool prof_on = false;
    long long prof_launches = 0;  // kernels enqueued during profiled steps
    long long steps_done = 0;     // host mirror of the step counter
    double time_host = 0.0;       // host mirror of the device time (same additions)
    Adj *adj = nullptr;
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? PIC_OK : PIC_ECUDA; }

void *dev_alloc(pic_s *h, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (h->alloc) p = h->alloc(bytes, h->ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) h->allocs.push_back(p);
    return p;
}

void dev_free(pic_s *h, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i] == p) {
            h->allocs.erase(h->allocs.begin() + i);
            break;
        }
    if (h->free) h->free(p, h->ctx);
    else cudaFree(p);
}

int bits_for(int n)
{
    int b = 1;
    while ((1 << b) < n) ++b;
    return b;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v)
{
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

int validate(const pic_config *c)
{
    if (!c || c->abi_version != PIC_ABI_VERSION) return PIC_EINVAL;
    const pic_grid &g = c->grid;
    if (g.dim != 2 && g.dim != 3) return PIC_EINVAL;
    if (c->shape_order < 1 || c->shape_order > 4) return PIC_EINVAL;
    double s = 0.0;
    long long ncell = 1;
    int bits = 0;
    for (int a = 0; a < g.dim; ++a) {
        if (g.n[a] < 4 || !(g.d[a] > 0.0)) return PIC_EINVAL;
        s += 1.0 / (g.d[a] * g.d[a]);
        ncell *= g.n[a];
        bits += bits_for(g.n[a]);
    }
    if (!(g.dt > 0.0) || g.dt * std::sqrt(s) >= 1.0) return PIC_EINVAL;  // Courant
    if (bits > 31 || ncell > 0x7fffffffLL) return PIC_EINVAL;
    if (g.bc_last != PIC_BC_PERIODIC && g.bc_last != PIC_BC_OPEN) return PIC_EINVAL;
    const int nl = g.n[g.dim - 1];
    const int margin = c->shape_order + 1;
    if (g.bc_last == PIC_BC_OPEN && nl < 2 * margin + 4) return PIC_EINVAL;
    if (c->n_species != 1 || !c->species) return PIC_EINVAL;
    const pic_species &sp = *c->species;
    if (!(sp.m > 0.0) || sp.q == 0.0) return PIC_EINVAL;
    if (c->laser.enabled) {
        const pic_laser &L = c->laser;
        if (L.plane < 1 || L.plane > nl - 2) return PIC_EINVAL;
        if (g.dim == 2 ? L.pol_axis != 0 : (L.pol_axis != 0 && L.pol_axis != 1)) return PIC_EINVAL;
        if (!(L.waist > 0.0) || !(L.fwhm > 0.0)) return PIC_EINVAL;
    }
    if (c->window.enabled) {
        if (g.bc_last != PIC_BC_OPEN || !(c->window.velocity > 0.0)) return PIC_EINVAL;
        for (int a = 0; a < g.dim; ++a)
            if (sp.ppc[a] < 1) return PIC_EINVAL;
        if (sp.n_knots > 0 && (!sp.profile_knots || !sp.per_particle_weight)) return PIC_EINVAL;
    }
    const pic_tuning &t = c->tuning;
    for (int a = 0; a < g.dim; ++a)
        if (t.tile[a] != 0 && !pow2(t.tile[a])) return PIC_EINVAL;
    if (t.drift < -1 || t.drift > 8) return PIC_EINVAL;
    if (t.block != 0 && t.block != 128 && t.block != 256 && t.block != 384 && t.block != 512) return PIC_EINVAL;
    if (t.sort_interval < 0) return PIC_EINVAL;
    if (t.sort_policy < 0 || t.sort_policy > 1) return PIC_EINVAL;
    if (t.persistent < 0 || t.persistent > 2) return PIC_EINVAL;
    if (t.stream_zero_tiles < 0 || t.stream_zero_tiles > 2) return PIC_EINVAL;
    if (t.deposit < 0 || t.deposit > 1 || (t.deposit == 1 && t.tma > 0)) return PIC_EINVAL;
    if (t.j_layout < 0 || t.j_layout > 1) return PIC_EINVAL;
    if (t.sort_rows < 0 || t.sort_rows > 2 || (t.sort_rows == 1 && t.sort_sub > 1)) return PIC_EINVAL;
    if (t.quiet_tiles < 0 || t.quiet_tiles > 2) return PIC_EINVAL;
    return PIC_OK;
}

int status_code(int bits)
{
    if (bits & kStatusOverflow) return PIC_EOVERFLOW;
    if (bits & kStatusTimeout) return PIC_ETIMEOUT;
    if (bits & kStatusBadIndex) return PIC_EINVAL;
    return PIC_OK;
}

int upload_runs(pic_s *h)
{
    std::vector<Run> tmp(h->nruns);
    for (int i = 0; i < h->nruns; ++i) tmp[i] = h->runs[i].r;
    cudaError_t e = cudaMemcpyAsync(h->d_runs, tmp.data(), sizeof(Run) * h->nruns, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_fail(e);
}

int set_seg(pic_s *h, int which, Seg &seg, const std::vector<long long> &items_per_run, int unit = kBlock)
{
    std::vector<int> start(h->nruns + 1, 0);
    for (int i = 0; i < h->nruns; ++i)
        start[i + 1] = start[i] + (int)((items_per_run[i] + unit - 1) / unit);
    int *dst = h->d_seg + which * (h->nruns + 1);
    cudaError_t e = cudaMemcpyAsync(dst, start.data(), sizeof(int) * (h->nruns + 1), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    seg.nruns = h->nruns;
    seg.start = dst;
    seg.nblocks = start[h->nruns];
    return cuda_fail(e);
}

// Allocate (or grow) the two particle buffers of run `hr` to `cap` slots,
// keeping the first `keep` slots of the current buffer.
int alloc_particles(pic_s *h, HostRun &hr, long long cap, long long keep, int cur_buf)
{
    Run &r = hr.r;
    const int dim = r.dim;
    const bool has_w = hr.sp.per_particle_weight != 0;
    const bool has_id = hr.cfg.track_ids != 0;
    ParticleBuf nb[2];
    for (int b = 0; b < 2; ++b) {
        std::memset(&nb[b], 0, sizeof(ParticleBuf));
        nb[b].cell = (int32_t *)dev_alloc(h, sizeof(int32_t) * cap);
        for (int a = 0; a < dim; ++a) nb[b].off[a] = (float *)dev_alloc(h, sizeof(float) * cap);
        for (int a = 0; a < 3; ++a) nb[b].u[a] = (float *)dev_alloc(h, sizeof(float) * cap);
        if (has_w) nb[b].w = (float *)dev_alloc(h, sizeof(float) * cap);
        if (has_id) nb[b].id = (int32_t *)dev_alloc(h, sizeof(int32_t) * cap);
        if (!nb[b].cell || !nb[b].u[2] || (has_w && !nb[b].w) || (has_id && !nb[b].id)) return PIC_ENOMEM;
        for (int a = 0; a < dim; ++a)
            if (!nb[b].off[a]) return PIC_ENOMEM;
    }
    if (keep > 0 && r.P[cur_buf].cell) {
        const ParticleBuf &o = r.P[cur_buf];
        ParticleBuf &n = nb[cur_buf];
        cudaError_t e = cudaSuccess;
        e = cudaMemcpyAsync(n.cell, o.cell, sizeof(int32_t) * keep, cudaMemcpyDeviceToDevice, h->stream);
        for (int a = 0; a < dim && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(n.off[a], o.off[a], sizeof(float) * keep, cudaMemcpyDeviceToDevice, h->stream);
        for (int a = 0; a < 3 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(n.u[a], o.u[a], sizeof(float) * keep, cudaMemcpyDeviceToDevice, h->stream);
        if (has_w && e == cudaSuccess)
            e = cudaMemcpyAsync(n.w, o.w, sizeof(float) * keep, cudaMemcpyDeviceToDevice, h->stream);
        if (has_id && e == cudaSuccess)
            e = cudaMemcpyAsync(n.id, o.id, sizeof(int32_t) * keep, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
    }
    for (int b = 0; b < 2; ++b) {
        ParticleBuf &o = r.P[b];
        if (o.cell) {
            dev_free(h, o.cell);
            for (int a = 0; a < dim; ++a) dev_free(h, o.off[a]);
            for (int a = 0; a < 3; ++a) dev_free(h, o.u[a]);
            dev_free(h, o.w);
            dev_free(h, o.id);
        }
        r.P[b] = nb[b];
    }
    r.capacity = cap;
    return PIC_OK;
}

int read_state(pic_s *h, int run, RunState *out)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, h->d_states + run, sizeof(RunState), cudaMemcpyDeviceToHost);
    return cuda_fail(e);
}

// Work items of the push kernel, largest expected cost first (the order in
// which the hardware or the persistent work queue hands them out): the
// slow-path tail blocks, then the tiles of runs with more particles per
// cell, then the rest.
int build_items(pic_s *h)
{
    std::vector<Item> items;
    // tail items of kTail particles, or larger ones when more than four per
    // SM would be needed (an item past the current tail returns at once, but
    // each still costs a CTA launch)
    long long tail_items = 0;
    for (int i = 0; i < h->nruns; ++i) {
        const HostRun &hr = h->runs[i];
        const long long max_tail = (long long)(h->sort_interval + 1) * hr.inject_per_shift;
        tail_items += (max_tail + kTail - 1) / kTail;
    }
    const long long cap = 4ll * (h->num_sms > 0 ? h->num_sms : 1);
    h->tail_block = tail_items > cap ? (int)(kTail * ((tail_items + cap - 1) / cap)) : kTail;
    for (int i = 0; i < h->nruns; ++i) {
        const HostRun &hr = h->runs[i];
        if (hr.inject_per_shift > 0) {
            const long long max_tail = (long long)(h->sort_interval + 1) * hr.inject_per_shift;
            const int tail_blocks = (int)((max_tail + h->tail_block - 1) / h->tail_block);
            for (int b = 0; b < tail_blocks; ++b) items.push_back(Item{i, 1, b, 0});
        }
    }
    const int n_tail = (int)items.size();
    std::vector<int> order(h->nruns);
    for (int i = 0; i < h->nruns; ++i) order[i] = i;
    auto load = [&](int i) {
        const Run &r = h->runs[i].r;
        return (long double)(r.capacity > 0 ? r.capacity : 1) / (long double)(r.ntiles > 0 ? r.ntiles : 1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return load(a) > load(b); });
    for (int i : order) {
        const HostRun &hr = h->runs[i];
        for (int t = 0; t < hr.r.ntiles; ++t) items.push_back(Item{i, 0, t, 0});
    }
    if (h->d_items) dev_free(h, h->d_items);
    if (h->d_live) dev_free(h, h->d_live);
    if (h->d_zero) dev_free(h, h->d_zero);
    if (h->d_nq) dev_free(h, h->d_nq);
    const size_t nb = sizeof(Item) * (items.size() ? items.size() : 1);
    h->d_items = (Item *)dev_alloc(h, nb);
    h->d_live = (Item *)dev_alloc(h, nb);
    h->d_zero = (Item *)dev_alloc(h, nb);
    h->d_nq = (Item *)dev_alloc(h, nb);  // (every tile of every run fits)
    if (!h->d_items || !h->d_live || !h->d_zero || !h->d_nq) return PIC_ENOMEM;
    // the field update walks the non-quiet tiles when every run keeps quiet
    // flags and 4-cell rows, and the handle is large enough for the three
    // extra launches per step to pay (below 2^22 cells a step takes tens of
    // microseconds and the cell kernels are faster)
    h->field_list = h->classify && h->yee_quad;
    long long cells = 0;
    for (int i = 0; i < h->nruns; ++i) {
        h->field_list = h->field_list && h->runs[i].r.quiet;
        cells += h->runs[i].r.ncell;
    }
    h->field_list = h->field_list && (h->quiet_mode == 1 || (h->quiet_mode == 0 && cells >= (1ll << 22)));
    h->n_items = (int)items.size();
    h->n_tail = n_tail;
    cudaError_t e = cudaMemcpyAsync(h->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice,
                                    h->stream);
    // the live list starts with the tail items; the classification appends the live tiles
    if (e == cudaSuccess && n_tail)
        e = cudaMemcpyAsync(h->d_live, items.data(), sizeof(Item) * n_tail, cudaMemcpyHostToDevice, h->stream);
    // the list of rows of tiles (along x) that are not quiet starts with every
    // row, so that the first J reset clears them all (each step's quiet
    // kernels then write the list the next J reset and that step's field
    // update walk)
    std::vector<Item> rows;
    for (int i = 0; i < h->nruns; ++i) {
        const Run &r = h->runs[i].r;
        const int nrows = r.nt[1] * (r.dim == 3 ? r.nt[2] : 1);
        for (int a = 0; a < nrows; ++a) rows.push_back(Item{i, 0, a, 0});
    }
    const int n_all = (int)rows.size();
    if (e == cudaSuccess && n_all > 0)
        e = cudaMemcpyAsync(h->d_nq, rows.data(), sizeof(Item) * n_all, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_cnt + 3, &n_all, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_fail(e);
}

// Mark every tile of run `hr` as possibly holding non-zero fields (after E or
// B was written from outside the timestep); the next second B half step
// recomputes the flags.
cudaError_t flag_all_tiles(pic_s *h, HostRun &hr)
{
    return hr.r.fz ? cudaMemsetAsync(hr.r.fz, 1, (size_t)hr.r.ntiles, h->stream) : cudaSuccess;
}

int enqueue_step(pic_s *h, bool sort, bool adaptive)
{
    cudaError_t e = cudaSuccess;
    const Run *R = h->d_runs;
    cudaStream_t st = h->stream;
    cudaEvent_t *ev = nullptr;
    if (h->prof_on && h->prof_steps < h->prof_max) ev = &h->prof_events[(size_t)h->prof_steps * kEvPerStep];
    auto mark = [&](int ph) {
        if (ev && e == cudaSuccess) e = cudaEventRecord(ev[ph], st);
    };
    mark(PIC_PH_SORT);
    // a recorded step keeps, after its sort, the slot each particle had before it
    int32_t *src_out = nullptr;
    if (sort && h->adj && h->adj->rec_on) src_out = h->adj->rec[h->steps_done - h->adj->rec_base].src;
    if (sort || adaptive)
        e = launch_sort(R, h->nruns, h->seg_parts, h->seg_keys, h->d_scan, src_out, sort ? 1 : 0, h->sort_interval,
                        adaptive ? 1 : 0, st);
    if (e == cudaSuccess && h->adj && h->adj->rec_on) {
        // the push of this step reads these particles and fields
        Rec &rc = h->adj->rec[h->steps_done - h->adj->rec_base];
        const Run &r0 = h->runs[0].r;
        rc.time = h->time_host;
        rc.sorted = sort;
        // one launch records particles, fields and tile offsets
        FieldCopy fc{};
        for (int c = 0; c < 3; ++c) {
            fc.src[c] = r0.E[c];
            fc.dst[c] = rc.E[c];
            fc.src[3 + c] = r0.B[c];
            fc.dst[3 + c] = rc.B[c];
        }
        fc.nf = 6;
        fc.cells = r0.ncell;
        fc.toff_src = r0.tile_off;
        fc.toff_dst = rc.tile_off;
        fc.nt = r0.ntiles + 1;
        e = launch_record(h->dim, R, rc.pc, h->adj->nslot, fc, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rc.st, h->d_states, sizeof(RunState), cudaMemcpyDeviceToDevice, st);
    }
    mark(PIC_PH_ZERO_J);
    // J is +0 outside the tiles that were not quiet at the last step
    if (e == cudaSuccess && h->field_list) e = launch_field_list(0, h->dim, R, h->d_nq, h->d_cnt + 3, 0, st);
    else if (e == cudaSuccess) e = launch_zero_j(R, h->seg_cells, h->yee_quad, st);
    mark(PIC_PH_PUSH);
    if (h->classify) {
        // live tiles (and the tail) through the staged kernel, zero-field tiles streamed
        const int n_tiles = h->n_items - h->n_tail;
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_cnt, 0, sizeof(int) * 4, st);
        if (e == cudaSuccess)
            e = launch_classify(R, h->d_items, h->n_tail, h->n_items, h->stage_lo, h->stage_len, h->d_live, h->d_zero,
                                h->d_cnt, st);
        const PushArgs a{R, h->d_live, h->n_tail, h->d_cnt, n_tiles, h->block, h->tail_block,
                         h->persistent ? h->d_cnt + 2 : nullptr, h->num_sms};
        if (e == cudaSuccess) e = launch_push(h->dim, h->order, h->tile, h->drift, h->variant(), a, st);
        if (ev && e == cudaSuccess) e = cudaEventRecord(ev[kMarkZero], st);
        if (e == cudaSuccess)
            e = launch_push_zero(h->dim, h->order, h->split, R, h->d_zero, h->d_cnt + 1, n_tiles, h->num_sms,
                                 h->zero_wide, st);
    } else {
        const PushArgs a{R, h->d_items, h->n_items, nullptr, 0, h->block, h->tail_block,
                         h->persistent ? h->d_queue : nullptr, h->num_sms};
        if (e == cudaSuccess) e = launch_push(h->dim, h->order, h->tile, h->drift, h->variant(), a, st);
        if (ev && e == cudaSuccess) e = cudaEventRecord(ev[kMarkZero], st);
    }
    mark(PIC_PH_YEE_B1);
    if (h->field_list) {  // quiet tiles: their field update is the identity; the others from a list
        if (e == cudaSuccess) e = launch_quiet(R, h->nruns, h->max_tiles, h->d_nq, h->d_cnt + 3, st);
        if (e == cudaSuccess) e = launch_field_list(1, h->dim, R, h->d_nq, h->d_cnt + 3, 0, st);
        mark(PIC_PH_YEE_E);
        if (e == cudaSuccess && h->any_open) e = launch_mur_save(R, h->seg_planes, st);
        if (e == cudaSuccess) e = launch_field_list(2, h->dim, R, h->d_nq, h->d_cnt + 3, 0, st);
        if (e == cudaSuccess && h->any_open) e = launch_mur_apply(R, h->seg_planes, st);
        mark(PIC_PH_YEE_B2);
        if (e == cudaSuccess) e = launch_field_list(1, h->dim, R, h->d_nq, h->d_cnt + 3, 1, st);
    } else {
        if (e == cudaSuccess) e = launch_yee_b(h->dim, R, h->seg_cells, 0, h->yee_quad, st);
        mark(PIC_PH_YEE_E);
        if (e == cudaSuccess && h->any_open) e = launch_mur_save(R, h->seg_planes, st);
        if (e == cudaSuccess) e = launch_yee_e(h->dim, R, h->seg_cells, h->yee_quad, st);
        if (e == cudaSuccess && h->any_open) e = launch_mur_apply(R, h->seg_planes, st);
        mark(PIC_PH_YEE_B2);
        if (e == cudaSuccess) e = launch_yee_b(h->dim, R, h->seg_cells, 1, h->yee_quad, st);
    }
    mark(PIC_PH_WINDOW);
    if (e == cudaSuccess) e = launch_end_step(R, h->nruns, st);
    if (e == cudaSuccess && h->any_window) e = launch_window(R, h->seg_planes, h->seg_inject, st);
    mark(kMarkEnd);
    if (ev) {
        h->prof_steps += 1;
        // sort 8, J reset 1, particle phase 1 (with the streaming: classification,
        // staged, streaming kernels and quiet tiles 4), Yee 3, end of step 1
        h->prof_launches += (sort || adaptive ? 8 : 0) + 1 + (h->classify ? 3 : 1) + (h->field_list ? 2 : 0) + 3 + 1 +
                            (h->any_open ? 2 : 0) + (h->any_window ? 3 : 0) + (h->adj && h->adj->rec_on ? 1 : 0);
    }
    return cuda_fail(e);
}

int first_step_setup(pic_s *h)
{
    std::vector<long long> parts(h->nruns), inj(h->nruns);
    for (int i = 0; i < h->nruns; ++i) {
        HostRun &hr = h->runs[i];
        hr.r.id_base = hr.loaded;  // the window's injected particles are numbered after the loaded ones
        if (!hr.r.P[0].cell) {  // never loaded: give it the injection room only
            long long cap = (long long)(h->sort_interval + 2) * hr.inject_per_shift + 4096;
            int rc = alloc_particles(h, hr, cap, 0, 0);
            if (rc) return rc;
        }
        parts[i] = hr.r.capacity;
        inj[i] = hr.inject_per_shift;
    }
    int rc = upload_runs(h);
    if (!rc) rc = set_seg(h, 2, h->seg_parts, parts, kSortChunk);
    if (!rc) {
        std::vector<long long> keys(h->nruns);
        for (int i = 0; i < h->nruns; ++i) keys[i] = (long long)h->runs[i].r.ntiles * h->runs[i].r.nsub;
        rc = set_seg(h, 4, h->seg_keys, keys, kScanChunk);
    }
    if (!rc && !h->d_scan) {
        h->d_scan = (int *)dev_alloc(h, sizeof(int) * (h->seg_keys.nblocks + 1));
        if (!h->d_scan) rc = PIC_ENOMEM;
    }
    if (!rc) rc = set_seg(h, 3, h->seg_inject, inj);
    if (!rc) rc = build_items(h);
    if (rc) return rc;
    h->zero_wide = true;
    for (int i = 0; i < h->nruns; ++i) {
        long long per_tile = 1;
        for (int a = 0; a < h->dim; ++a) per_tile *= (long long)h->tile[a] * h->runs[i].sp.ppc[a];
        h->zero_wide = h->zero_wide && per_tile >= 4096;
    }
    // the initial electron charge is the neutralising background (rho_0)
    for (int i = 0; i < h->nruns; ++i) {
        HostRun &hr = h->runs[i];
        cudaError_t e = cudaMemsetAsync(hr.r.rho0, 0, sizeof(double) * hr.r.ncell, h->stream);
        if (e == cudaSuccess) e = launch_charge(h->dim, h->order, h->d_runs + i, hr.r.rho0, hr.r.capacity, h->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
    }
    // sets the push kernel's shared-memory limit outside any graph capture
    const PushArgs a0{h->d_runs, h->d_items, 0, nullptr, 0, h->block, kTail, nullptr, 1};
    cudaError_t e = launch_push(h->dim, h->order, h->tile, h->drift, h->variant(), a0, h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    h->started = true;
    return PIC_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// TMA tensor maps of the six field components for the push kernel's 3D
// field tile (one box per component and tile), when TMA staging is on.
// Left null (the kernel then stages with plain loads) when a field base or
// row is not on a 16-byte boundary.
int build_tensor_maps(pic_s *h, HostRun &hr)
{
    Run &r = hr.r;
    r.tmap = nullptr;
    int box[3] = {0, 0, 0};
    if (r.dim != 3 || !h->use_tma || !push_tma_box(3, h->order, h->tile, h->drift, box)) return PIC_OK;
    if ((r.n[0] * sizeof(float)) % 16 != 0) return PIC_OK;
    EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return PIC_OK;
    CUtensorMap maps[6];
    const cuuint64_t dims[3] = {(cuuint64_t)r.n[0], (cuuint64_t)r.n[1], (cuuint64_t)r.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)r.n[0] * sizeof(float), (cuuint64_t)r.n[0] * r.n[1] * sizeof(float)};
    const cuuint32_t bx[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]}, es[3] = {1, 1, 1};
    for (int c = 0; c < 6; ++c) {
        void *base = c < 3 ? (void *)r.E[c] : (void *)r.B[c - 3];
        if ((uintptr_t)base % 16 != 0) return PIC_OK;
        if (enc(&maps[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return PIC_OK;
    }
    void *d = dev_alloc(h, sizeof(maps));
    if (!d) return PIC_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(d, maps, sizeof(maps), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    r.tmap = d;
    return PIC_OK;
}

int init_run(pic_s *h, HostRun &hr, int idx)
{
    const pic_config &c = hr.cfg;
    Run &r = hr.r;
    std::memset(&r, 0, sizeof(Run));
    r.dim = c.grid.dim;
    r.order = c.shape_order;
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        r.n[a] = a < r.dim ? c.grid.n[a] : 1;
        r.d[a] = a < r.dim ? (float)c.grid.d[a] : 1.f;
        r.inv_d[a] = (float)(1.0 / (a < r.dim ? c.grid.d[a] : 1.0));
        r.dt_over_d[a] = (float)(c.grid.dt / (a < r.dim ? c.grid.d[a] : 1.0));
        r.d_over_dt[a] = (float)((a < r.dim ? c.grid.d[a] : 1.0) / c.grid.dt);
        r.bits[a] = a < r.dim ? bits_for(r.n[a]) : 0;
        int T = a < r.dim ? h->tile[a] : 1;
        r.tlog[a] = ilog2(T);
        r.nt[a] = a < r.dim ? (r.n[a] + T - 1) / T : 1;
        ncell *= r.n[a];
    }
    r.ncell = (int)ncell;
    r.ntiles = r.nt[0] * r.nt[1] * r.nt[2];
    r.dt = (float)c.grid.dt;
    r.dt_d = c.grid.dt;
    r.d_last_d = c.grid.d[c.grid.dim - 1];
    for (int a = 0; a < 3; ++a) r.dd[a] = a < r.dim ? c.grid.d[a] : 1.0;
    r.q = (float)hr.sp.q;
    r.m = (float)hr.sp.m;
    r.qm_half_dt = (float)(0.5 * hr.sp.q / hr.sp.m * c.grid.dt);
    r.w_const = (float)hr.sp.w_const;
    r.open_last = c.grid.bc_last == PIC_BC_OPEN;
    r.margin = r.open_last ? c.shape_order + 1 : 0;
    r.drift = h->drift;
    const int nl = r.n[r.dim - 1];
    const int plane = (int)(ncell / nl);
    r.jst = h->j4 ? 4 : 1;
    float *j4 = h->j4 ? (float *)dev_alloc(h, sizeof(float) * 4 * ncell) : nullptr;
    for (int a = 0; a < 3; ++a) {
        r.E[a] = (float *)dev_alloc(h, sizeof(float) * ncell);
        r.B[a] = (float *)dev_alloc(h, sizeof(float) * ncell);
        r.J[a] = h->j4 ? (j4 ? j4 + a : nullptr) : (float *)dev_alloc(h, sizeof(float) * ncell);
        if (!r.E[a] || !r.B[a] || !r.J[a]) return PIC_ENOMEM;
    }
    r.rho0 = (double *)dev_alloc(h, sizeof(double) * ncell);
    hr.rho = (double *)dev_alloc(h, sizeof(double) * ncell);
    hr.rho32 = (float *)dev_alloc(h, sizeof(float) * ncell);
    r.mur = (float *)dev_alloc(h, sizeof(float) * 8 * plane);
    r.tile_off = (int32_t *)dev_alloc(h, sizeof(int32_t) * (r.ntiles + 1));
    r.nsub = h->sort_sub;
    r.sort_rows = h->sort_rows ? 1 : 0;
    if (r.sort_rows) r.nsub = 1 << (r.tlog[1] + (r.dim == 3 ? r.tlog[2] : 0));  // rows of cells along x
    if ((long long)r.ntiles * r.nsub > (1ll << 30)) return PIC_EINVAL;
    r.tile_cnt = (int32_t *)dev_alloc(h, sizeof(int32_t) * ((size_t)r.ntiles * r.nsub + 1));
    r.fz = (uint8_t *)dev_alloc(h, (size_t)r.ntiles);
    if (!r.rho0 || !hr.rho || !hr.rho32 || !r.mur || !r.tile_off || !r.tile_cnt || !r.fz) return PIC_ENOMEM;
    if (h->classify && h->quiet_mode != 2) {  // quiet tiles: the field update skips them (with the zero-field streaming)
        static const int kDepositReach[5] = {0, 2, 3, 3, 4};  // cells beyond a particle's cell its window reaches
        for (int a = 0; a < 3; ++a) {
            // (a particle may be a drift allowance, or one move, from its tile)
            const int T = 1 << r.tlog[a], reach = (r.drift > 1 ? r.drift : 1) + kDepositReach[r.order];
            r.qr[a] = a < r.dim ? (reach + T - 1) / T : 0;
        }
        r.jt = (uint8_t *)dev_alloc(h, (size_t)r.ntiles);
        r.quiet = (uint8_t *)dev_alloc(h, (size_t)r.ntiles);
        if (!r.jt || !r.quiet) return PIC_ENOMEM;
        if (cudaMemsetAsync(r.jt, 0, (size_t)r.ntiles, h->stream) != cudaSuccess ||
            cudaMemsetAsync(r.quiet, 0, (size_t)r.ntiles, h->stream) != cudaSuccess)
            return PIC_ECUDA;
    }
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        e = cudaMemsetAsync(r.E[a], 0, sizeof(float) * ncell, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.B[a], 0, sizeof(float) * ncell, h->stream);
        if (e == cudaSuccess && (!h->j4 || a == 0))
            e = cudaMemsetAsync(r.J[a], 0, sizeof(float) * ncell * r.jst, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(r.rho0, 0, sizeof(double) * ncell, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.mur, 0, sizeof(float) * 8 * plane, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.tile_off, 0, sizeof(int32_t) * (r.ntiles + 1), h->stream);
    // E = B = +0 in every tile; loading a moving particle flags its tile
    // (pack_kernel), writing E or B flags every tile
    if (e == cudaSuccess) e = cudaMemsetAsync(r.fz, 0, (size_t)r.ntiles, h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    const pic_laser &L = c.laser;
    r.laser_on = L.enabled;
    r.laser_pol = L.pol_axis;
    r.laser_plane = L.plane;
    r.a0 = L.a0;
    r.omega0 = L.omega0;
    r.waist = L.waist;
    r.fwhm = L.fwhm;
    r.t_peak = L.t_peak;
    r.window_on = c.window.enabled;
    r.window_v = c.window.velocity;
    r.window_t0 = c.window.t_start;
    for (int a = 0; a < 3; ++a) r.ppc[a] = a < r.dim ? hr.sp.ppc[a] : 1;
    r.density = hr.sp.density;
    r.n_knots = hr.sp.n_knots;
    r.z0 = hr.sp.profile_z0;
    r.z1 = hr.sp.profile_z1;
    if (hr.sp.n_knots > 0 && hr.sp.profile_knots) {
        hr.knots.assign(hr.sp.profile_knots, hr.sp.profile_knots + hr.sp.n_knots);
        double *dk = (double *)dev_alloc(h, sizeof(double) * hr.sp.n_knots);
        if (!dk) return PIC_ENOMEM;
        e = cudaMemcpyAsync(dk, hr.knots.data(), sizeof(double) * hr.sp.n_knots, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
        r.knots = dk;
    }
    hr.inject_per_shift = 0;
    if (r.window_on) {
        long long ppc_t = (long long)r.ppc[0] * r.ppc[1] * (r.dim == 3 ? r.ppc[2] : 1);
        hr.inject_per_shift = (long long)plane * ppc_t;
    }
    r.state = h->d_states + idx;
    return build_tensor_maps(h, hr);
}

int create_common(const pic_config *cfgs, int n, pic_t **out)
{
    if (!out || !cfgs || n < 1) return PIC_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        int rc = validate(&cfgs[i]);
        if (rc) return rc;
        if (cfgs[i].grid.dim != cfgs[0].grid.dim || cfgs[i].shape_order != cfgs[0].shape_order) return PIC_EINVAL;
    }
    pic_s *h = new (std::nothrow) pic_s();
    if (!h) return PIC_ENOMEM;
    const pic_config &c0 = cfgs[0];
    h->nruns = n;
    h->dim = c0.grid.dim;
    h->order = c0.shape_order;
    h->stream = (cudaStream_t)c0.stream;
    h->alloc = c0.alloc;
    h->free = c0.free;
    h->ctx = c0.alloc_ctx;
    const pic_tuning &t = c0.tuning;
    for (int a = 0; a < 3; ++a) {
        int def = h->dim == 3 ? 8 : 16;
        h->tile[a] = a < h->dim ? (t.tile[a] ? t.tile[a] : def) : 1;
    }
    h->drift = t.drift >= 0 ? t.drift : push_default_drift(h->dim, h->tile);
    h->block = t.block ? t.block : (h->dim == 3 ? 512 : 256);
    h->sort_adaptive = t.sort_policy == 0;
    // sort_interval: the longest interval of the adaptive policy (also what
    // the injection room and tail items are sized for); fixed_interval: the
    // interval of the fixed schedule, which the adjoint form uses as well
    h->fixed_interval = t.sort_interval ? t.sort_interval : 4;
    h->sort_interval = t.sort_interval ? t.sort_interval : (h->sort_adaptive ? kSortMaxAdaptive : 4);
    h->use_graph = t.use_graph != 0 && h->stream != nullptr;
    h->persistent = t.persistent == 1 || (t.persistent == 0 && n > 1);
    h->sort_sub = t.sort_sub ? t.sort_sub : 1;
    h->sort_rows = t.sort_rows == 1 || (t.sort_rows == 0 && h->sort_sub == 1);
    h->quiet_mode = t.quiet_tiles;
    h->use_tma = t.tma > 0;
    h->split = t.deposit == 1;
    h->j4 = t.j_layout == 1;
    h->adjoint_keep = t.adjoint_keep;
    h->classify = t.stream_zero_tiles != 2;
    if (h->sort_sub < 1 || h->sort_sub > 32 || (h->sort_sub & (h->sort_sub - 1))) {
        delete h;
        return PIC_EINVAL;
    }
    h->push_smem = push_smem_bytes(h->dim, h->order, h->tile, h->drift, h->variant());
    if (h->push_smem == 0 ||  // (tile, drift) not among the compiled configurations
        !push_stage_extent(h->dim, h->order, h->tile, h->drift, h->variant(), h->stage_lo, h->stage_len)) {
        delete h;
        return PIC_EINVAL;
    }
    int dev = 0;
    int max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        delete h;
        return PIC_ECUDA;
    }
    if (h->push_smem + sizeof(Run) + 512 > (size_t)max_smem) {  // + the kernels' static shared memory
        delete h;
        return PIC_EINVAL;  // tile + halo does not fit in shared memory
    }
    h->runs.resize(n);
    h->d_runs = (Run *)dev_alloc(h, sizeof(Run) * n);
    h->d_states = (RunState *)dev_alloc(h, sizeof(RunState) * n);
    h->d_seg = (int *)dev_alloc(h, sizeof(int) * 5 * (n + 1));
    h->d_diag = (double *)dev_alloc(h, sizeof(double) * 16);
    h->d_count = (unsigned long long *)dev_alloc(h, sizeof(unsigned long long));
    h->d_queue = (int *)dev_alloc(h, sizeof(int));
    h->d_cnt = (int *)dev_alloc(h, sizeof(int) * 4);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (!h->d_runs || !h->d_states || !h->d_seg || !h->d_diag || !h->d_count || !h->d_queue || !h->d_cnt) {
        pic_destroy(h);
        return PIC_ENOMEM;
    }
    if (cudaMemsetAsync(h->d_states, 0, sizeof(RunState) * n, h->stream) != cudaSuccess) {
        pic_destroy(h);
        return PIC_ECUDA;
    }
    std::vector<long long> cells(n), planes(n);
    for (int i = 0; i < n; ++i) {
        HostRun &hr = h->runs[i];
        hr.cfg = cfgs[i];
        hr.sp = *cfgs[i].species;
        hr.cfg.species = &hr.sp;
        int rc = init_run(h, hr, i);
        if (rc) {
            pic_destroy(h);
            return rc;
        }
        cells[i] = hr.r.ncell;
        planes[i] = hr.r.ncell / hr.r.n[hr.r.dim - 1];
        h->any_open = h->any_open || hr.r.open_last;
        h->any_window = h->any_window || hr.r.window_on;
        h->max_tiles = hr.r.ntiles > h->max_tiles ? hr.r.ntiles : h->max_tiles;
        bool aligned = hr.r.n[0] % 4 == 0;
        for (int c = 0; c < 3; ++c)
            aligned = aligned && (uintptr_t)hr.r.E[c] % 16 == 0 && (uintptr_t)hr.r.B[c] % 16 == 0 &&
                      (uintptr_t)hr.r.J[hr.r.jst == 4 ? 0 : c] % 16 == 0;
        h->yee_quad = h->yee_quad && aligned;
        // a configured capacity is allocated now (the loads then only copy)
        if (hr.cfg.capacity > 0) {
            rc = alloc_particles(h, hr, hr.cfg.capacity, 0, 0);
            if (rc) {
                pic_destroy(h);
                return rc;
            }
        }
    }
    int rc = upload_runs(h);
    if (!rc) rc = set_seg(h, 0, h->seg_cells, cells);
    if (!rc) rc = set_seg(h, 1, h->seg_planes, planes);
    if (rc) {
        pic_destroy(h);
        return rc;
    }
    *out = h;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_create(const pic_config *cfg, pic_t **out) { return create_common(cfg, 1, out); }

int pic_create_batch(const pic_config *cfgs, int32_t n, pic_t **out) { return create_common(cfgs, n, out); }

int pic_select_run(pic_t *h, int32_t run)
{
    if (!h || run < 0 || run >= h->nruns) return PIC_EINVAL;
    h->cur = run;
    return PIC_OK;
}

int32_t pic_num_runs(const pic_t *h) { return h ? h->nruns : 0; }

int pic_load_particles(pic_t *h, int32_t species, int64_t n, const int32_t *cell, const float *off, const float *u,
                       const float *w)
{
    if (!h || species != 0 || n < 0) return PIC_EINVAL;
    if (h->started) return PIC_ESTATE;
    if (n == 0) return PIC_OK;
    if (!cell || !off || !u) return PIC_EINVAL;
    HostRun &hr = h->runs[h->cur];
    if (hr.sp.per_particle_weight && !w) return PIC_EINVAL;
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    const long long have = st.n_total;
    const long long need = have + n;
    const long long room = (long long)(h->sort_interval + 2) * hr.inject_per_shift + 4096;
    if (!hr.r.P[0].cell || need + room > hr.r.capacity) {
        if (hr.cfg.capacity > 0 && need + room > hr.cfg.capacity && hr.r.P[0].cell) return PIC_EOVERFLOW;
        long long cap = hr.cfg.capacity > 0 ? hr.cfg.capacity : (long long)(need * 1.25) + room;
        if (cap < need + room) cap = need + room;
        rc = alloc_particles(h, hr, cap, have, st.buf);
        if (rc) return rc;
        rc = upload_runs(h);
        if (rc) return rc;
    }
    const int dim = hr.r.dim;
    // stage the host arrays on the device, then pack into the current buffer
    size_t bytes = sizeof(int32_t) * dim * n + sizeof(float) * dim * n + sizeof(float) * 3 * n +
                   (w ? sizeof(float) * n : 0);
    char *stage = (char *)dev_alloc(h, bytes + 1024);
    if (!stage) return PIC_ENOMEM;
    int32_t *dc = (int32_t *)stage;
    float *doff = (float *)(dc + (size_t)dim * n);
    float *du = doff + (size_t)dim * n;
    float *dw = w ? du + (size_t)3 * n : nullptr;
    cudaError_t e = cudaMemcpyAsync(dc, cell, sizeof(int32_t) * dim * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off, sizeof(float) * dim * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(du, u, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync(dw, w, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_pack(h->d_runs + h->cur, have, n, dim, dc, doff, du, dw, h->stream);
    if (e == cudaSuccess) e = launch_set_count(h->d_runs + h->cur, need, 0, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, stage);
    hr.loaded = need;
    if (e != cudaSuccess) return PIC_ECUDA;
    if (cudaMemcpy(&st, h->d_states + h->cur, sizeof(RunState), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PIC_ECUDA;
    h->need_sort = true;
    return status_code(st.status);
}

int pic_step(pic_t *h, int32_t nsteps)
{
    if (!h || nsteps < 0) return PIC_EINVAL;
    if (!h->started) {
        int rc = first_step_setup(h);
        if (rc) return rc;
    }
    if (h->adj && h->adj->spent) return PIC_ESTATE;
    for (int s = 0; s < nsteps; ++s) {
        if (h->adj && h->adj->save_ckpt) {  // forward run: record the kept segments
            Adj &a = *h->adj;
            a.rec_on = a.keep > 0 && h->steps_done >= a.keep_base && h->steps_done < a.total;
            a.rec_base = a.keep_base;
        }
        if (h->adj && h->adj->save_ckpt && h->steps_done % h->adj->K == 0 &&
            h->steps_done / h->adj->K < h->adj->nck) {
            Ckpt &ck = h->adj->ck[h->steps_done / h->adj->K];
            const Run &r0 = h->runs[0].r;
            cudaError_t e = launch_part_copy(h->dim, h->d_runs, ck.pc, h->adj->nslot, 0, h->stream);
            for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
                e = cudaMemcpyAsync(ck.E[c], r0.E[c], sizeof(float) * r0.ncell, cudaMemcpyDeviceToDevice, h->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(ck.B[c], r0.B[c], sizeof(float) * r0.ncell, cudaMemcpyDeviceToDevice,
                                        h->stream);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ck.st, h->d_states, sizeof(RunState), cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return PIC_ECUDA;
            ck.time = h->time_host;
        }
        // adaptive policy: the device decides each step (sort_decide_kernel);
        // the host forces a sort only where it must (after loads, at the start
        // of a recomputed segment).  The adjoint keeps the fixed schedule, so
        // that a recomputed segment repeats the forward run's sorts.
        const bool adaptive = h->sort_adaptive && !h->adj;
        bool sort = h->need_sort || (!adaptive && h->since_sort >= h->fixed_interval);
        int kind = (sort ? 1 : 0) + (adaptive ? 2 : 0);
        if (h->use_graph && !h->prof_on && !(h->adj && h->adj->rec_on)) {
            if (!h->graph[kind]) {
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PIC_ECUDA;
                int rc = enqueue_step(h, sort, adaptive);
                cudaError_t e = cudaStreamEndCapture(h->stream, &g);
                if (rc || e != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return rc ? rc : PIC_ECUDA;
                }
                e = cudaGraphInstantiate(&h->graph[kind], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return PIC_ECUDA;
            }
            if (cudaGraphLaunch(h->graph[kind], h->stream) != cudaSuccess) return PIC_ECUDA;
        } else {
            int rc = enqueue_step(h, sort, adaptive);
            if (rc) return rc;
        }
        if (sort) {
            h->need_sort = false;
            h->since_sort = 0;
        }
        h->since_sort += 1;
        h->steps_done += 1;
        h->time_host += h->runs[0].cfg.grid.dt;
    }
    return PIC_OK;
}

int pic_sync(pic_t *h)
{
    if (!h) return PIC_EINVAL;
    int worst = PIC_OK;
    for (int i = 0; i < h->nruns; ++i) {
        RunState st;
        int rc = read_state(h, i, &st);
        if (rc) return rc;
        int c = status_code(st.status);
        if (c) worst = c;
    }
    return worst;
}

static int copy_field(pic_t *h, const HostRun &hr, const RunState &st, float *arr, float *ext, bool to_ext,
                      int on_device)
{
    const Run &r = hr.r;
    const int nl = r.n[r.dim - 1];
    const size_t plane = (size_t)r.ncell / nl;
    const int o = r.open_last ? st.origin : 0;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (to_ext ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
    // window frame index p <-> storage (p + origin) mod nl: two contiguous slabs
    size_t a_n = (size_t)(nl - o) * plane, b_n = (size_t)o * plane;
    cudaError_t e;
    if (to_ext) {
        e = cudaMemcpyAsync(ext, arr + (size_t)o * plane, sizeof(float) * a_n, kind, h->stream);
        if (e == cudaSuccess && b_n) e = cudaMemcpyAsync(ext + a_n, arr, sizeof(float) * b_n, kind, h->stream);
    } else {
        e = cudaMemcpyAsync(arr + (size_t)o * plane, ext, sizeof(float) * a_n, kind, h->stream);
        if (e == cudaSuccess && b_n) e = cudaMemcpyAsync(arr, ext + a_n, sizeof(float) * b_n, kind, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_fail(e);
}

int pic_read_fields(pic_t *h, int32_t which, float *dst, size_t n_elems, int32_t on_device)
{
    if (!h || !dst || which < 0 || which > PIC_RHO) return PIC_EINVAL;
    HostRun &hr = h->runs[h->cur];
    if (n_elems < (size_t)hr.r.ncell) return PIC_EINVAL;
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    float *src = nullptr;
    if (which < 3) src = hr.r.E[which];
    else if (which < 6) src = hr.r.B[which - 3];
    else if (which < 9 && hr.r.jst == 1) src = hr.r.J[which - 6];
    else if (which < 9) {  // one lane of the four-component nodes, gathered into the FP32 scratch
        cudaError_t e = cudaMemcpy2DAsync(hr.rho32, sizeof(float), hr.r.J[which - 6], 4 * sizeof(float),
                                          sizeof(float), (size_t)hr.r.ncell, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
        src = hr.rho32;
    } else {
        if (!h->started) {
            int r2 = upload_runs(h);
            if (r2) return r2;
        }
        cudaError_t e = cudaMemsetAsync(hr.rho, 0, sizeof(double) * hr.r.ncell, h->stream);
        if (e == cudaSuccess && hr.r.P[0].cell)
            e = launch_charge(h->dim, h->order, h->d_runs + h->cur, hr.rho, hr.r.capacity, h->stream);
        if (e == cudaSuccess) e = launch_to_float(hr.rho, hr.rho32, hr.r.ncell, h->stream);
        if (e != cudaSuccess) return PIC_ECUDA;
        src = hr.rho32;
    }
    rc = copy_field(h, hr, st, src, dst, true, on_device);
    if (rc) return rc;
    return status_code(st.status);
}

int pic_write_fields(pic_t *h, int32_t which, const float *src, size_t n_elems, int32_t on_device)
{
    if (!h || !src || which < 0 || which > PIC_BZ) return PIC_EINVAL;
    HostRun &hr = h->runs[h->cur];
    if (n_elems < (size_t)hr.r.ncell) return PIC_EINVAL;
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    float *dstp = which < 3 ? hr.r.E[which] : hr.r.B[which - 3];
    if (flag_all_tiles(h, hr) != cudaSuccess) return PIC_ECUDA;
    return copy_field(h, hr, st, dstp, const_cast<float *>(src), false, on_device);
}

int pic_read_particles(pic_t *h, int32_t species, int32_t *cell, float *off, float *u, float *w, int32_t *id,
                       int64_t cap, int64_t *n)
{
    if (!h || species != 0 || cap < 0 || !n) return PIC_EINVAL;
    HostRun &hr = h->runs[h->cur];
    *n = 0;
    if (!hr.r.P[0].cell) return PIC_OK;
    if (!h->started) {
        int rc = upload_runs(h);
        if (rc) return rc;
    }
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    const int dim = hr.r.dim;
    const long long slots = st.n_total;
    const long long m = slots > 0 ? slots : 1;
    size_t bytes = (sizeof(int32_t) * dim + sizeof(float) * dim + sizeof(float) * 4 + sizeof(int32_t)) * (size_t)m;
    char *stage = (char *)dev_alloc(h, bytes + 1024);
    if (!stage) return PIC_ENOMEM;
    int32_t *dc = (int32_t *)stage;
    float *doff = (float *)(dc + (size_t)dim * m);
    float *du = doff + (size_t)dim * m;
    float *dw = du + (size_t)3 * m;
    int32_t *did = (int32_t *)(dw + m);
    cudaError_t e = cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = launch_unpack(h->d_runs + h->cur, m, dim, dc, doff, du, dw, did, h->d_count, h->stream);
    unsigned long long cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, h->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        dev_free(h, stage);
        return PIC_ECUDA;
    }
    *n = (int64_t)cnt;
    if ((long long)cnt > cap) {
        dev_free(h, stage);
        return PIC_EOVERFLOW;
    }
    for (int a = 0; a < dim && e == cudaSuccess; ++a) {
        if (cell) e = cudaMemcpyAsync(cell + (size_t)a * cap, dc + (size_t)a * m, sizeof(int32_t) * cnt,
                                      cudaMemcpyDeviceToHost, h->stream);
        if (off && e == cudaSuccess)
            e = cudaMemcpyAsync(off + (size_t)a * cap, doff + (size_t)a * m, sizeof(float) * cnt,
                                cudaMemcpyDeviceToHost, h->stream);
    }
    for (int a = 0; a < 3 && u && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(u + (size_t)a * cap, du + (size_t)a * m, sizeof(float) * cnt, cudaMemcpyDeviceToHost,
                            h->stream);
    if (w && e == cudaSuccess) e = cudaMemcpyAsync(w, dw, sizeof(float) * cnt, cudaMemcpyDeviceToHost, h->stream);
    if (id && e == cudaSuccess) e = cudaMemcpyAsync(id, did, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, stage);
    if (e != cudaSuccess) return PIC_ECUDA;
    return status_code(st.status);
}

int pic_diagnostics(pic_t *h, pic_diag *out)
{
    if (!h || !out) return PIC_EINVAL;
    std::memset(out, 0, sizeof(*out));
    HostRun &hr = h->runs[h->cur];
    if (!h->started) {
        int rc = upload_runs(h);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemsetAsync(h->d_diag, 0, sizeof(double) * 16, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hr.rho, 0, sizeof(double) * hr.r.ncell, h->stream);
    if (e == cudaSuccess && hr.r.P[0].cell)
        e = launch_charge(h->dim, h->order, h->d_runs + h->cur, hr.rho, hr.r.capacity, h->stream);
    if (e == cudaSuccess) e = launch_diag(h->dim, h->d_runs + h->cur, hr.rho, hr.r.capacity, h->d_diag, h->stream);
    double dd[16];
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, h->d_diag, sizeof(dd), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    const Run &r = hr.r;
    const double V = (double)r.d[0] * r.d[1] * (r.dim == 3 ? r.d[2] : 1.0);
    unsigned um[4];
    std::memcpy(um, dd + 8, sizeof(um));
    float mres, mrho;
    std::memcpy(&mres, &um[0], 4);
    std::memcpy(&mrho, &um[1], 4);
    out->step = st.step;
    out->time = st.time;
    out->shifts = st.shifts;
    out->W_E = 0.5 * dd[0] * V;
    out->W_B = 0.5 * dd[1] * V;
    out->W_kin = dd[2] * V;
    out->n_particles = (int64_t)dd[3];
    out->gauss_resid = mrho > 0.f ? (double)mres / (double)mrho : (double)mres;
    out->imbalance = (um[3] > 0 && dd[3] > 0) ? (double)um[2] / (dd[3] / (double)um[3]) : 0.0;
    out->slow_path = (int64_t)st.slow_last;
    out->sorts = (int32_t)st.sorts;
    out->streamed = (int64_t)st.streamed;
    out->live_tiles = (int64_t)st.live_tiles;
    out->status = status_code(st.status);
    return out->status;
}

int pic_profile_begin(pic_t *h, int32_t max_steps)
{
    if (!h || max_steps < 1) return PIC_EINVAL;
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    h->prof_events.assign((size_t)max_steps * kEvPerStep, nullptr);
    for (auto &ev : h->prof_events)
        if (cudaEventCreate(&ev) != cudaSuccess) return PIC_ECUDA;
    h->prof_max = max_steps;
    h->prof_steps = 0;
    h->prof_launches = 0;
    h->prof_on = true;
    return PIC_OK;
}

int pic_profile_end(pic_t *h, double *ms, int32_t n_phases, int64_t *launches)
{
    if (!h || !h->prof_on || !ms || n_phases < 1) return PIC_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PIC_ECUDA;
    const int np = n_phases < PIC_NUM_PHASES ? n_phases : PIC_NUM_PHASES;
    for (int p = 0; p < n_phases; ++p) ms[p] = 0.0;
    for (int s = 0; s < h->prof_steps; ++s) {
        cudaEvent_t *ev = &h->prof_events[(size_t)s * kEvPerStep];
        for (int p = 0; p < np; ++p) {
            float t = 0.f;
            cudaError_t e = p == PIC_PH_PUSH_ZERO ? cudaEventElapsedTime(&t, ev[kMarkZero], ev[PIC_PH_YEE_B1])
                                                  : cudaEventElapsedTime(&t, ev[p], ev[p + 1]);
            if (e != cudaSuccess) return PIC_ECUDA;
            ms[p] += t;
        }
    }
    if (launches) *launches = h->prof_launches;
    h->prof_on = false;
    return PIC_OK;
}

int pic_adjoint_begin(pic_t *h, int32_t total_steps, int32_t checkpoint_every)
{
    if (!h || total_steps < 1 || checkpoint_every < 1) return PIC_EINVAL;
    if (h->started || h->adj || h->nruns != 1) return PIC_ESTATE;
    HostRun &hr = h->runs[0];
    if (!hr.cfg.track_ids || !hr.sp.per_particle_weight || hr.loaded <= 0) return PIC_EINVAL;
    if (h->order > 3) return PIC_EINVAL;  // (the reverse kernels are compiled for orders 1 to 3)
    if (h->split) return PIC_EINVAL;      // (they transpose the undivided deposit)
    RunState st;
    int rc = read_state(h, 0, &st);
    if (rc) return rc;
    if (st.n_total <= 0) return PIC_EINVAL;
    Run &r = hr.r;
    // ids: the loaded particles, and with a moving window the layers it can
    // inject during the run; slots: with a window every slot of the buffers
    const long long n0 = st.n_total;
    long long nid = n0, nslot = n0;
    if (r.window_on) {
        const double travel = r.window_v * (st.time + (double)total_steps * r.dt_d - r.window_t0);
        const long long max_shifts = travel > 0.0 ? (long long)(travel / r.d_last_d) + 2 : 0;
        nid = n0 + max_shifts * hr.inject_per_shift;
        nslot = r.capacity;
        if (nid >= 2147483647ll) return PIC_EINVAL;  // (ids are int32)
    }
    Adj *a = new (std::nothrow) Adj();
    if (!a) return PIC_ENOMEM;
    h->adj = a;
    const long long n = nslot, nc = r.ncell;
    const int dim = r.dim;
    a->K = checkpoint_every;
    a->total = total_steps;
    a->nck = (total_steps + checkpoint_every - 1) / checkpoint_every;
    a->nid = nid;
    a->nslot = nslot;
    a->nload = n0;
    auto F = [&](long long cnt) { return (float *)dev_alloc(h, sizeof(float) * cnt); };
    bool ok = true;
    for (int c = 0; c < 3; ++c) {
        a->A.lE[c] = F(nc);
        a->A.lB[c] = F(nc);
        a->A.lJ[c] = F(nc);
        a->A.T[c] = F(nc);
        a->A.nE[c] = F(nc);
        a->A.lu[c] = F(nid);
        a->A.lx[c] = c < dim ? F(nid) : nullptr;
        a->A.su[c] = F(n);
        a->A.sx[c] = c < dim ? F(n) : nullptr;
        a->A.ou[c] = F(n);
        a->A.ox[c] = c < dim ? F(n) : nullptr;
        ok = ok && a->A.lE[c] && a->A.lB[c] && a->A.lJ[c] && a->A.T[c] && a->A.nE[c] && a->A.lu[c] &&
             (c >= dim || a->A.lx[c]) && a->A.su[c] && (c >= dim || a->A.sx[c]) && a->A.ou[c] &&
             (c >= dim || a->A.ox[c]);
    }
    a->A.lw = (double *)dev_alloc(h, sizeof(double) * nid);
    a->A.sw = (double *)dev_alloc(h, sizeof(double) * n);
    a->A.ow = (double *)dev_alloc(h, sizeof(double) * n);
    ok = ok && a->A.sw && a->A.ow;
    a->A.wid = F(nid);
    a->zb = F(nid);
    a->la0 = (double *)dev_alloc(h, sizeof(double) * 4);
    a->red = (double *)dev_alloc(h, sizeof(double) * 4);
    a->dk = (double *)dev_alloc(h, sizeof(double) * 1024);
    ok = ok && a->A.lw && a->A.wid && a->zb && a->la0 && a->red && a->dk;
    auto part = [&](bool with_w) {
        PartCopy pc{};
        pc.cell = (int32_t *)dev_alloc(h, sizeof(int32_t) * n);
        for (int c = 0; c < dim; ++c) pc.off[c] = F(n);
        for (int c = 0; c < 3; ++c) pc.u[c] = F(n);
        pc.w = with_w ? F(n) : nullptr;
        pc.id = (int32_t *)dev_alloc(h, sizeof(int32_t) * n);
        ok = ok && pc.cell && pc.id && pc.u[2] && (!with_w || pc.w);
        for (int c = 0; c < dim; ++c) ok = ok && pc.off[c];
        return pc;
    };
    a->ck.resize(a->nck);
    for (Ckpt &ck : a->ck) {
        ck.pc = part(true);
        for (int c = 0; c < 3; ++c) {
            ck.E[c] = F(nc);
            ck.B[c] = F(nc);
            ok = ok && ck.E[c] && ck.B[c];
        }
        ck.st = (RunState *)dev_alloc(h, sizeof(RunState));
        ok = ok && ck.st;
    }
    auto record = [&]() {
        Rec rc2{};
        rc2.pc = part(true);
        rc2.tile_off = (int32_t *)dev_alloc(h, sizeof(int32_t) * (r.ntiles + 1));
        rc2.src = (int32_t *)dev_alloc(h, sizeof(int32_t) * n);
        rc2.st = (RunState *)dev_alloc(h, sizeof(RunState));
        bool good = rc2.tile_off && rc2.src && rc2.st && rc2.pc.cell && rc2.pc.id && rc2.pc.u[2];
        for (int c = 0; c < 3; ++c) {
            rc2.E[c] = F(nc);
            rc2.B[c] = F(nc);
            good = good && rc2.E[c] && rc2.B[c];
        }
        return std::make_pair(rc2, good);
    };
    for (int q = 0; q < a->K && ok; ++q) {
        auto rg = record();
        a->rec.push_back(rg.first);
        ok = ok && rg.second;
    }
    if (!ok) return PIC_ENOMEM;
    // Segments kept from the forward run (their records are taken while it
    // runs, so the reverse sweep does not recompute them): as many as the
    // request allows and 75 % of the free device memory holds.
    const int req = h->adjoint_keep;
    int keep = req < 0 ? 0 : (req == 0 ? a->nck : (req < a->nck ? req : a->nck));
    if (keep > 1) {
        size_t fr = 0, tot = 0;
        const size_t rec_bytes = sizeof(int32_t) * (size_t)n * 3 + sizeof(float) * (size_t)n * (dim + 4) +
                                 sizeof(float) * 6 * (size_t)nc + sizeof(int32_t) * (r.ntiles + 1) + 6 * 256;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
        const long long fit = (long long)(0.75 * (double)fr / ((double)rec_bytes * a->K));
        keep = (int)(keep - 1 < fit ? keep : fit + 1);
    }
    for (int q = a->K; q < keep * a->K; ++q) {
        auto rg = record();
        if (!rg.second) {  // keep what fitted (whole segments)
            keep = q / a->K;
            break;
        }
        a->rec.push_back(rg.first);
    }
    a->keep = keep;
    a->keep_base = (a->nck - keep) * a->K;
    r.id_base = n0;  // (as the first step sets it)
    r.adj_zb = a->zb;
    r.adj_nid = nid;
    rc = upload_runs(h);
    if (rc) return rc;
    cudaError_t e = launch_adj_init(h->d_runs, a->A.wid, a->zb, n, nid, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    // checkpoints are taken between graph replays; the recording steps of
    // the reverse sweep run without graphs (their record buffers change)
    return PIC_OK;
}

static int objective_reduce(pic_t *h, const pic_objective *obj, double *L)
{
    if (!h || !obj || !L || !(obj->width > 0.0)) return PIC_EINVAL;
    if (!h->started) {
        int rc = first_step_setup(h);
        if (rc) return rc;
    }
    HostRun &hr = h->runs[0];
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    double *red = h->adj ? h->adj->red : h->d_diag;
    const ObjArgs o{(float)obj->z_lo, (float)obj->z_hi, (float)obj->width};
    AdjPtrs none{};
    cudaError_t e = cudaMemsetAsync(red, 0, sizeof(double) * 2, h->stream);
    if (e == cudaSuccess)
        e = launch_objective(h->d_runs + h->cur, st.origin, o, red, hr.r.capacity, 0, none, h->stream);
    double hv[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv, red, sizeof(hv), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return PIC_ECUDA;
    *L = hv[1] > 0.0 ? hv[0] / hv[1] : 0.0;
    return PIC_OK;
}

int pic_objective_value(pic_t *h, const pic_objective *obj, double *L)
{
    return objective_reduce(h, obj, L);
}

int pic_adjoint_kept(pic_t *h)
{
    if (!h || !h->adj) return PIC_ESTATE;
    return h->adj->keep;
}

int pic_adjoint_backward(pic_t *h, const pic_objective *obj, double *L, double *dL_da0, double *dL_dknots,
                         int32_t n_knots, double *dL_dw)
{
    if (!h || !h->adj || h->adj->spent) return PIC_ESTATE;
    Adj &a = *h->adj;
    if (h->steps_done != a.total) return PIC_ESTATE;
    if (n_knots < 0 || n_knots > 1024 || (n_knots > 0 && !dL_dknots)) return PIC_EINVAL;
    HostRun &hr = h->runs[0];
    const Run &r = hr.r;
    double Lv = 0.0;
    int rc = objective_reduce(h, obj, &Lv);
    if (rc) return rc;
    if (L) *L = Lv;
    const long long n = a.nslot, nid = a.nid, nc = r.ncell;
    const int dim = r.dim;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemsetAsync(a.A.lE[c], 0, sizeof(float) * nc, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.A.lB[c], 0, sizeof(float) * nc, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.A.lu[c], 0, sizeof(float) * nid, st);
        if (e == cudaSuccess && c < dim) e = cudaMemsetAsync(a.A.lx[c], 0, sizeof(float) * nid, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(a.A.lw, 0, sizeof(double) * nid, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.la0, 0, sizeof(double), st);
    const ObjArgs o{(float)obj->z_lo, (float)obj->z_hi, (float)obj->width};
    RunState cur;
    rc = read_state(h, 0, &cur);
    if (rc) return rc;
    if (e == cudaSuccess) e = launch_objective(h->d_runs, cur.origin, o, a.red, r.capacity, 1, a.A, st);
    if (e != cudaSuccess) return PIC_ECUDA;
    const int plane = r.ncell / r.n[dim - 1];
    a.rec_on = false;
    // window shifts: the step before a record whose shift count is larger
    // ended with a shift (at most one per step)
    int next_shifts = cur.shifts;
    std::vector<RunState> hst(a.K);
    for (int seg = a.nck - 1; seg >= 0; --seg) {
        const int s0 = seg * a.K, s1 = s0 + a.K < a.total ? s0 + a.K : a.total;
        const bool kept = seg >= a.nck - a.keep;  // recorded by the forward run
        const int rb = kept ? a.keep_base : s0;   // step of record 0
        Ckpt &ck = a.ck[seg];
        if (!kept) {
        // restore the segment's start state and recompute it, recording each step
        e = cudaMemcpyAsync(h->d_states, ck.st, sizeof(RunState), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = launch_part_copy(h->dim, h->d_runs, ck.pc, n, 1, st);
        for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
            e = cudaMemcpyAsync(r.E[c], ck.E[c], sizeof(float) * nc, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r.B[c], ck.B[c], sizeof(float) * nc, cudaMemcpyDeviceToDevice, st);
        }
        if (e == cudaSuccess) e = flag_all_tiles(h, h->runs[0]);
        if (e != cudaSuccess) return PIC_ECUDA;
        h->steps_done = s0;
        h->time_host = ck.time;
        h->need_sort = true;
        a.save_ckpt = false;
        a.rec_on = true;
        a.rec_base = s0;
        rc = pic_step(h, s1 - s0);
        a.rec_on = false;
        if (rc) return rc;
        }
        // the run states the segment's pushes started from (origin, slot counts)
        for (int s = s0; s < s1 && e == cudaSuccess; ++s)
            e = cudaMemcpyAsync(&hst[s - s0], a.rec[s - rb].st, sizeof(RunState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        // particle adjoints follow the slot order of each record: they move to
        // the slots before a sort through the sort's record of them, and
        // through id order at segment ends
        for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
            e = cudaMemsetAsync(a.A.su[c], 0, sizeof(float) * n, st);
            if (e == cudaSuccess && c < dim) e = cudaMemsetAsync(a.A.sx[c], 0, sizeof(float) * n, st);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(a.A.sw, 0, sizeof(double) * n, st);
        if (e == cudaSuccess) e = launch_adj_perm(dim, a.A, a.rec[s1 - 1 - rb].pc.id, n, nid, 1, st);
        if (e != cudaSuccess) return PIC_ECUDA;
        for (int s = s1 - 1; s >= s0; --s) {
            const Rec &rc2 = a.rec[s - rb];
            const RunState &rs = hst[s - s0];
            if (next_shifts > rs.shifts) {
                // the step ended with a window shift: zeroed front plane (storage
                // index = this step's origin) and an injected layer appended at
                // slot rs.n_total; inside the segment its slot adjoints go to id
                // order here, at the segment's last step they are there already
                e = launch_adj_window(a.A, plane, rs.origin, s < s1 - 1 ? rs.n_total : -1, hr.inject_per_shift,
                                      r.id_base + (long long)(next_shifts - 1) * hr.inject_per_shift, nid, st);
                if (e != cudaSuccess) return PIC_ECUDA;
            }
            next_shifts = rs.shifts;
            e = launch_adj_fields(dim, h->d_runs, a.A, (int)nc, plane, rs.origin, rc2.time, r.dt_d, r.laser_on, a.la0,
                                  st);
            TrajStep ts{};
            ts.cell = rc2.pc.cell;
            for (int c = 0; c < 3; ++c) {
                ts.off[c] = rc2.pc.off[c];
                ts.u[c] = rc2.pc.u[c];
                ts.E[c] = rc2.E[c];
                ts.B[c] = rc2.B[c];
            }
            ts.id = rc2.pc.id;
            ts.w = rc2.pc.w;
            ts.tile_off = rc2.tile_off;
            ts.n = n;
            ts.first = 0;
            // after a sort inside the segment the kernel writes the adjoints at
            // the slots of the previous record (zero for particles the sort dropped)
            const bool moved = s > s0 && rc2.sorted;
            ts.src = moved ? rc2.src : nullptr;
            for (int c = 0; c < 3 && moved && e == cudaSuccess; ++c) {
                e = cudaMemsetAsync(a.A.ou[c], 0, sizeof(float) * n, st);
                if (e == cudaSuccess && c < dim) e = cudaMemsetAsync(a.A.ox[c], 0, sizeof(float) * n, st);
            }
            if (e == cudaSuccess && moved) e = cudaMemsetAsync(a.A.ow, 0, sizeof(double) * n, st);
            if (e == cudaSuccess) e = launch_adj_particles(dim, r.order, h->d_runs, r, a.A, ts, rs.origin, st);
            if (e == cudaSuccess && rs.n_total > rs.n_sorted) {
                // the unsorted tail (particles the window injected since the
                // last sort), pushed by the tail items in the forward step
                TrajStep tt = ts;
                tt.tile_off = nullptr;
                tt.first = rs.n_sorted;
                tt.n = rs.n_total;
                e = launch_adj_particles(dim, r.order, h->d_runs, r, a.A, tt, rs.origin, st);
            }
            if (moved) {
                for (int c = 0; c < 3; ++c) {
                    std::swap(a.A.sx[c], a.A.ox[c]);
                    std::swap(a.A.su[c], a.A.ou[c]);
                }
                std::swap(a.A.sw, a.A.ow);
            }
            // the segment's first record: back to id order for the previous segment
            if (e == cudaSuccess && s == s0) e = launch_adj_perm(dim, a.A, rc2.pc.id, n, nid, 0, st);
            if (e != cudaSuccess) return PIC_ECUDA;
        }
    }
    a.spent = true;  // the handle now holds a recomputed intermediate state
    double la0 = 0.0;
    e = cudaMemcpyAsync(&la0, a.la0, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n_knots > 0) {
        e = cudaMemsetAsync(a.dk, 0, sizeof(double) * n_knots, st);
        const double ppc_t = (double)r.ppc[0] * r.ppc[1] * (dim == 3 ? r.ppc[2] : 1);
        if (e == cudaSuccess)
            e = launch_knots(a.A.lw, a.zb, nid, n_knots, hr.sp.profile_z0, hr.sp.profile_z1, ppc_t, a.dk, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dL_dknots, a.dk, sizeof(double) * n_knots, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && dL_dw)
        e = cudaMemcpyAsync(dL_dw, a.A.lw, sizeof(double) * a.nload, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return PIC_ECUDA;
    if (dL_da0) *dL_da0 = la0;
    return PIC_OK;
}

int pic_adjoint_particles(pic_t *h, float *lam_x, float *lam_u, const float *lam_j, double *lam_w, float *lam_f,
                          int64_t n)
{
    if (!h || !lam_x || !lam_u || !lam_j || !lam_w || !lam_f || n < 1) return PIC_EINVAL;
    if (h->nruns != 1) return PIC_ESTATE;
    HostRun &hr = h->runs[0];
    if (!hr.cfg.track_ids || !hr.sp.per_particle_weight || hr.r.window_on || h->order > 3 || h->split ||
        hr.loaded <= 0)
        return PIC_EINVAL;
    if (!h->started) {
        int rc = first_step_setup(h);
        if (rc) return rc;
    }
    RunState st;
    int rc = read_state(h, 0, &st);
    if (rc) return rc;
    const Run &r = hr.r;
    const int dim = r.dim;
    const long long ns = st.n_total, nc = r.ncell;
    if (ns < 1) return PIC_EINVAL;
    std::vector<void *> bufs;
    bool ok = true;
    auto F = [&](long long cnt) {
        void *p = dev_alloc(h, sizeof(float) * (size_t)cnt);
        ok = ok && p;
        bufs.push_back(p);
        return (float *)p;
    };
    auto D = [&](long long cnt) {
        void *p = dev_alloc(h, sizeof(double) * (size_t)cnt);
        ok = ok && p;
        bufs.push_back(p);
        return (double *)p;
    };
    AdjPtrs A{};
    for (int c = 0; c < 3; ++c) {
        A.lE[c] = F(nc);
        A.lB[c] = F(nc);
        A.lJ[c] = F(nc);
        A.lu[c] = F(n);
        A.su[c] = F(ns);
        if (c < dim) {
            A.lx[c] = F(n);
            A.sx[c] = F(ns);
        }
    }
    A.lw = D(n);
    A.sw = D(ns);
    cudaError_t e = ok ? cudaSuccess : cudaErrorMemoryAllocation;
    cudaStream_t s = h->stream;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemsetAsync(A.lE[c], 0, sizeof(float) * nc, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(A.lB[c], 0, sizeof(float) * nc, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(A.lJ[c], lam_j + c * nc, sizeof(float) * nc, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(A.lu[c], lam_u + c * n, sizeof(float) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && c < dim)
            e = cudaMemcpyAsync(A.lx[c], lam_x + c * n, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(A.lw, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.sw, 0, sizeof(double) * ns, s);
    const ParticleBuf &pb = r.P[st.buf];
    // adjoints by id -> by slot, the flat reverse kernel over every slot, back by id
    if (e == cudaSuccess) e = launch_adj_perm(dim, A, pb.id, ns, n, 1, s);
    TrajStep ts{};
    ts.cell = pb.cell;
    for (int c = 0; c < 3; ++c) {
        ts.off[c] = c < dim ? pb.off[c] : nullptr;
        ts.u[c] = pb.u[c];
        ts.E[c] = r.E[c];
        ts.B[c] = r.B[c];
    }
    ts.w = pb.w;
    ts.id = pb.id;
    ts.n = ns;
    if (e == cudaSuccess) e = launch_adj_particles(dim, h->order, h->d_runs, r, A, ts, 0, s);
    if (e == cudaSuccess) e = launch_adj_perm(dim, A, pb.id, ns, n, 0, s);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemcpyAsync(lam_f + c * nc, A.lE[c], sizeof(float) * nc, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lam_f + (3 + c) * nc, A.lB[c], sizeof(float) * nc, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lam_u + c * n, A.lu[c], sizeof(float) * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && c < dim)
            e = cudaMemcpyAsync(lam_x + c * n, A.lx[c], sizeof(float) * n, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam_w, A.lw, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (void *p : bufs) dev_free(h, p);
    if (!ok) return PIC_ENOMEM;
    return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_adjoint_fields(pic_t *h, float *lam, float *lam_j, double t)
{
    if (!h || !lam) return PIC_EINVAL;
    if (!h->started) {
        int rc = first_step_setup(h);
        if (rc) return rc;
    }
    HostRun &hr = h->runs[h->cur];
    const Run &r = hr.r;
    const size_t nc = (size_t)r.ncell;
    RunState st;
    int rc = read_state(h, h->cur, &st);
    if (rc) return rc;
    std::vector<float *> bufs;
    AdjPtrs A{};
    bool ok = true;
    auto F = [&]() {
        float *p = (float *)dev_alloc(h, sizeof(float) * nc);
        ok = ok && p;
        bufs.push_back(p);
        return p;
    };
    for (int c = 0; c < 3; ++c) {
        A.lE[c] = F();
        A.lB[c] = F();
        A.lJ[c] = F();
        A.T[c] = F();
        A.nE[c] = F();
    }
    double *la0 = (double *)dev_alloc(h, sizeof(double));
    cudaError_t e = (ok && la0) ? cudaSuccess : cudaErrorMemoryAllocation;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemcpyAsync(A.lE[c], lam + c * nc, sizeof(float) * nc, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(A.lB[c], lam + (3 + c) * nc, sizeof(float) * nc, cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(la0, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = launch_adj_fields(r.dim, h->d_runs + h->cur, A, (int)nc, (int)(nc / r.n[r.dim - 1]), st.origin, t,
                              r.dt_d, r.laser_on && st.shifts == 0, la0, h->stream);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemcpyAsync(lam + c * nc, A.lE[c], sizeof(float) * nc, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lam + (3 + c) * nc, A.lB[c], sizeof(float) * nc, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && lam_j)
            e = cudaMemcpyAsync(lam_j + c * nc, A.lJ[c], sizeof(float) * nc, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (float *p : bufs) dev_free(h, p);
    dev_free(h, la0);
    if (!ok) return PIC_ENOMEM;
    return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

void pic_destroy(pic_t *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    for (int k = 0; k < 4; ++k)
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    std::vector<void *> all = h->allocs;
    for (void *p : all) {
        if (h->free) h->free(p, h->ctx);
        else cudaFree(p);
    }
    delete h->adj;
    delete h;
}

const char *pic_strerror(int status)
{
    switch (status) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "device allocation failed";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_EOVERFLOW: return "particle capacity exceeded";
    case PIC_ETIMEOUT: return "bounded device wait gave up";
    case PIC_ESTATE: return "call not valid in the current state";
    default: return "unknown status";
    }
}

}  // extern "C"
