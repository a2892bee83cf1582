// internal.h -- host-side launchers of the device kernels (not part of the
// public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pic {

struct Run;
struct RunState;
struct Item;

// Segmented 1-D launches over several runs: block b belongs to the run r with
// start[r] <= b < start[r+1]; runs are located by binary search.
struct Seg {
    int nruns;
    const int *start;  // device array [nruns + 1]
    int nblocks;
};

constexpr int kBlock = 256;

// Tile sort (sort.cu): one CTA of kSortThreads threads ranks a chunk of
// kSortChunk particle slots in a shared-memory key table of kSortHash
// entries; the particle segments of the sort are in units of chunks.
constexpr int kSortThreads = 256, kSortItems = 8, kSortChunk = kSortThreads * kSortItems;
constexpr int kSortHashLog = 9, kSortHash = 1 << kSortHashLog, kSortProbe = 32;
// adaptive sort: sort once strays (particles outside their tile's drift
// region) add up to n_total / kSortSlowDiv particle-steps since the last sort
constexpr unsigned long long kSortSlowDiv = 65536;
// ... or once the unsorted tail the window injected holds n_total / kSortTailDiv
constexpr unsigned long long kSortTailDiv = 64;
// The exclusive scan of the (tile, sub-bucket) counters runs in blocks of
// kScanChunk keys (kScanThreads threads x kScanItems consecutive keys).
constexpr int kScanThreads = 256, kScanItems = 16, kScanChunk = kScanThreads * kScanItems;

// Particle kernel (push.cuh) over the compiled tile menu (push_menu.h).
// push_smem_bytes returns 0 for a (tile, drift) pair that is not compiled.
int push_default_drift(int dim, const int *tile);
// variant: 0 = field tile staged by plain loads, 1 = staged by TMA (3D
// only), 2 = plain staging with the virtual-trajectory deposit (the default
// tiles, orders 1-3)
size_t push_smem_bytes(int dim, int order, const int *tile, int drift, int variant);
// 3D: extents of the TMA box that loads one component of the field tile
// (returns 0 for 2D or an entry not compiled with TMA staging)
int push_tma_box(int dim, int order, const int *tile, int drift, int *box);
// the field region a tile stages: lo[a] cells before the tile origin, len[a]
// cells long, per axis (returns 0 for an entry that is not compiled)
int push_stage_extent(int dim, int order, const int *tile, int drift, int variant, int *lo, int *len);

// One launch of the staged particle kernel.
struct PushArgs {
    const Run *runs;
    const Item *items;
    int nitems;           // items of the launch; with live_cnt, the leading fixed items
    const int *live_cnt;  // device count of the items after the fixed ones (may be null)
    int max_extra;        // upper bound of that count
    int block, tail_block;
    int *queue;           // non-null: persistent grid of persistent_ctas x (CTAs per SM)
                          // taking items from this device counter (reset by the launch)
    int persistent_ctas;
};
cudaError_t launch_push(int dim, int order, const int *tile, int drift, int variant, const PushArgs &a,
                        cudaStream_t st);

// Per-step tile classification (push.cu): the tile items items[n_tail,
// n_items) are split into live tiles, appended to `live` after its n_tail
// tail items (count in cnt[0]), and zero-field tiles, written to `zero`
// (count in cnt[1]); cnt must be cleared before.  The zero-field tiles are
// then advanced by the streaming kernel (launch_push_zero).
cudaError_t launch_classify(const Run *runs, const Item *items, int n_tail, int n_items, const int *stage_lo,
                            const int *stage_len, Item *live, Item *zero, int *cnt, cudaStream_t st);
// wide: every run's tiles hold at least 4096 particles (four groups of four
// slots per thread and two CTAs per SM; otherwise two groups, three CTAs)
cudaError_t launch_push_zero(int dim, int order, bool split, const Run *runs, const Item *zero, const int *count,
                             int max_items, int num_sms, bool wide, cudaStream_t st);

// fields.cu
cudaError_t launch_zero_j(const Run *runs, Seg cells, bool quad, cudaStream_t st);
// quad: four x cells per thread with 16-byte accesses (every run's n0 a
// multiple of 4 and its field arrays 16-byte aligned)
cudaError_t launch_yee_b(int dim, const Run *runs, Seg cells, int second_half, bool quad, cudaStream_t st);
cudaError_t launch_yee_e(int dim, const Run *runs, Seg cells, bool quad, cudaStream_t st);
cudaError_t launch_mur_save(const Run *runs, Seg planes, cudaStream_t st);
cudaError_t launch_mur_apply(const Run *runs, Seg planes, cudaStream_t st);
cudaError_t launch_end_step(const Run *runs, int nruns, cudaStream_t st);
// quiet tiles of this step (after the particle phase, before the field
// update): the quiet flags, the list of the rows of tiles along x holding a
// tile that is not quiet (nq, Item::a = ty + nt[1] tz; count in *nq_count,
// which the caller zeroes first), then the step's tile flags cleared
cudaError_t launch_quiet(const Run *runs, int nruns, int max_tiles, Item *nq, int *nq_count, cudaStream_t st);
// the field update over the rows of tiles of a list: which 0 = J reset, 1 = B
// half step (second: the step's second half), 2 = E step; 4-cell rows only
cudaError_t launch_field_list(int which, int dim, const Run *runs, const Item *nq, const int *nq_count, int second,
                              cudaStream_t st);
cudaError_t launch_window(const Run *runs, Seg planes, Seg inject, cudaStream_t st);

// sort.cu
// keys: segments of kScanChunk (tile, sub-bucket) keys; scan_sums: one int
// per key block.
// src_out (may be null): for each sorted slot, the slot the particle had
// before the sort (single-run handles).
// force: every run sorts; adaptive: a run also sorts when max_interval
// steps have passed or its slow path has grown (sort_decide_kernel).
cudaError_t launch_sort(const Run *runs, int nruns, Seg parts, Seg keys, int *scan_sums, int32_t *src_out,
                        int force, int max_interval, int adaptive, cudaStream_t st);

// diag.cu
cudaError_t launch_pack(const Run *run, long long base, long long n, int dim, const int32_t *cell,
                        const float *off, const float *u, const float *w, cudaStream_t st);
cudaError_t launch_set_count(const Run *run, long long n_total, int sorted, cudaStream_t st);
// charge density of the live particles accumulated in FP64 (diagnostics only)
cudaError_t launch_charge(int dim, int order, const Run *run, double *rho, long long cap, cudaStream_t st);
cudaError_t launch_to_float(const double *src, float *dst, long long n, cudaStream_t st);
cudaError_t launch_unpack(const Run *run, long long cap, int dim, int32_t *cell, float *off, float *u, float *w,
                          int32_t *id, unsigned long long *count, cudaStream_t st);
// out (16 doubles): [0] sum E^2, [1] sum B^2, [2] sum w m (gamma - 1), [3] live particles;
// out+8 viewed as unsigned[4]: max|div E - (rho - rho0)| and max|rho0| (float bits of the
// FP64 values rounded down to FP32),
// max particles in a tile, occupied tiles.
cudaError_t launch_diag(int dim, const Run *run, const double *rho, long long cap, double *out, cudaStream_t st);

// adjoint.cu -- reverse sweep of the timestep
struct AdjPtrs {
    float *lE[3], *lB[3], *lJ[3], *T[3], *nE[3];  // field adjoints and scratch
    float *lx[3], *lu[3];                         // particle adjoints by id
    double *lw;                                   // dL/dw by id
    float *wid;                                   // weight by id
    float *sx[3], *su[3];                         // particle adjoints by slot of the current record
    double *sw;
    float *ox[3], *ou[3];                         // the same, permuted to the slots before a sort
    double *ow;
};
// one recorded step: the particles and fields the push of that step read
struct TrajStep {
    const int32_t *cell;
    const float *off[3];
    const float *u[3];
    const float *w;
    const int32_t *id;
    const int32_t *tile_off;  // tile offsets of the sort these slots follow (null: flat kernel)
    const int32_t *src;       // slot each particle had before the sort of this step (null: no sort);
                              // outputs then go to ox/ou/ow at that slot
    long long n;
    long long first;  // flat kernel: slots [first, n)
    const float *E[3];
    const float *B[3];
};
struct ObjArgs {
    float z_lo, z_hi, width;
};
// (the lamE and newE scratch buffers of A trade places)
cudaError_t launch_adj_fields(int dim, const Run *run, AdjPtrs &A, int ncell, int plane, int origin, double t_n,
                              double dt, int laser_on, double *la0, cudaStream_t st);
cudaError_t launch_adj_particles(int dim, int order, const Run *run, const Run &host_run, const AdjPtrs &A,
                                 const TrajStep &ts, int origin, cudaStream_t st);
// seed == 0: reduce sum w K sigma and sum w sigma into red[0..1]; seed == 1: seed the adjoints
cudaError_t launch_objective(const Run *run, int origin, const ObjArgs &o, double *red, long long cap, int seed,
                             const AdjPtrs &A, cudaStream_t st);
cudaError_t launch_knots(const double *lw, const float *zb, long long n, int n_knots, double z0, double z1,
                         double ppc_t, double *out, cudaStream_t st);
// n: particle slots to read, nid: ids the arrays hold
cudaError_t launch_adj_init(const Run *run, float *wid, float *zb, long long n, long long nid, cudaStream_t st);
struct PartCopy {
    int32_t *cell;
    float *off[3];
    float *u[3];
    float *w;    // may be null
    int32_t *id; // may be null
};
cudaError_t launch_part_copy(int dim, const Run *run, const PartCopy &pc, long long n, int restore, cudaStream_t st);
// Extra arrays copied by the same launch as a particle record (may be empty):
// nf field arrays of `cells` floats and `nt` ints of tile offsets.
struct FieldCopy {
    const float *src[6];
    float *dst[6];
    int nf;
    long long cells;
    const int32_t *toff_src;
    int32_t *toff_dst;
    long long nt;
};
cudaError_t launch_record(int dim, const Run *run, const PartCopy &pc, long long n, const FieldCopy &fc,
                          cudaStream_t st);
// move the particle adjoints between id order and the slot order of a record
// slot adjoints of n slots to (to_slots = 0) or from (1) id order, ids < nid
cudaError_t launch_adj_perm(int dim, const AdjPtrs &A, const int32_t *id, long long n, long long nid, int to_slots,
                            cudaStream_t st);
// transpose of a window shift: field adjoints zeroed on storage plane
// store_plane of the last axis (plane cells each); the injected layer at
// slots slot0 .. slot0+count-1 (ids id0 + j) moved to id order (slot0 < 0: skip)
cudaError_t launch_adj_window(const AdjPtrs &A, int plane, int store_plane, long long slot0, long long count,
                              long long id0, long long nid, cudaStream_t st);

}  // namespace pic
