// ljmd_api.cu -- host side of the C ABI declared in include/ljmd.h.
//
// Owns the device memory of a box (through the installed allocator hook),
// orders its work on an internal stream fenced against the caller's stream,
// and replays the velocity-Verlet step loop from captured CUDA graphs.  Each
// graph holds `chunk` steps; between graphs the host reads the device error
// word once, so a neighbour-list overflow found inside a graph is repaired by
// restoring the state saved before that graph, regrowing the list and
// replaying it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ljmd.h"
#include "ljmd_internal.cuh"

namespace {

md_alloc_fn g_alloc = nullptr;
md_free_fn g_free = nullptr;
void* g_ctx = nullptr;

struct Alloc {
    void* p;
    size_t bytes;
};

struct GraphEnt {
    int64_t nsteps;
    double dt;
    int energy;
    cudaGraphExec_t exec;
    int64_t kernels;                 // kernel nodes per replay
    std::vector<cudaEvent_t> ev;     // phase events (profiling), 8 per step
    std::vector<char> used;          // which (step, phase) pairs were recorded
};

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int round_up(int64_t x, int64_t m) { return (int)(((x + m - 1) / m) * m); }

}  // namespace

struct md_box {
    int device = 0;
    int nsm = 152;
    cudaStream_t ustream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    // the energy reduction's branch of the step graph (it overlaps the list update)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the rebuild sequence as the body of a conditional (IF) graph node
    bool use_cond = false;   // list update as a conditional graph node (md_set_graph_conditional)
    cudaStream_t cstream = nullptr;            // captures the node's body
    unsigned long long* d_cond_runs = nullptr; // true conditions so far (device)
    unsigned long long cond_runs_seen = 0;
    md_alloc_fn alloc = nullptr;
    md_free_fn free_ = nullptr;
    void* actx = nullptr;
    int prec = 0;
    int nrep = 0;
    int64_t ntot = 0;
    int np = 0;
    std::vector<RepDev> reps;
    std::vector<int4> chunks;
    std::vector<int4> titems;   // energy-reduction items
    std::vector<int4> tiles;
    std::vector<int4> segs;
    // LJ
    bool lj_set = false;
    int nt = 1;
    double skin = 0.0, rl = 0.0;
    bool fresh_abs = true;     // xabs holds the current positions (slot order)
    bool binned = false;       // cell ids and offsets are valid
    // device
    BoxDev d{};
    RepDev* d_rep = nullptr;
    int4* d_chunk = nullptr;
    int4* d_seg = nullptr;
    LJDev* d_lj = nullptr;
    int4* d_tiles = nullptr;
    std::vector<int4> bricks;  // work items of the tiled force kernel: (replica, first cell x, y, z)
    size_t pf_cap = 0;         // doubles of d.part_f
    int4* d_brick = nullptr;
    int* d_tile_sum = nullptr;
    int* d_type_user = nullptr;
    double* d_thermo = nullptr;
    int64_t thermo_cap = 0;    // doubles
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    std::vector<Alloc> allocs;
    // snapshot of the step-loop state (list overflow repair)
    std::vector<std::pair<void*, size_t>> snap_src;
    void* d_snap = nullptr;
    size_t snap_bytes = 0;
    // graphs
    std::vector<GraphEnt> graphs;
    int64_t chunk_steps = 100;
    // all-pairs form and thermostat
    bool all_pairs = false;
    double tstat_rate = 0.0;
    double* d_tstat_T = nullptr;
    long long* d_step_ctr = nullptr;
    // tuning
    int min_capacity = 0;
    bool autofit = false;      // fit the capacity after the next full build
    double cell_scale = 1.0;   // cell edge / list radius (>= 1)
    int list_kernel = 0;       // MD_LIST_AUTO / MD_LIST_QUADS / MD_LIST_LANES
    int force_kernel = 0;      // MD_FORCE_AUTO / MD_FORCE_CHUNKS / MD_FORCE_TILES
    int order = 0;             // order inside a cell (MD_ORDER_*)
    int force_per_sm = 0;      // 0 = automatic (tuning)
    int list_per_sm = 0;
    int seg_cells = 0;
    int64_t steps = 0;
    int64_t launches = 0;
    bool profiling = false;
    double prof_ms[4] = {0, 0, 0, 0};
    int64_t prof_n[4] = {0, 0, 0, 0};
    // recorded forward run (md_integrate with ckpt_every > 0)
    bool rec_valid = false;
    int64_t rec_serial = 0;    // serial number of the last recorded run
    int64_t rec_nsteps = 0;
    int rec_k = 0, rec_C = 0;
    double rec_dt = 0.0;
    std::vector<std::pair<void*, size_t>> ck_src;   // arrays saved per checkpoint
    char* d_ckpt = nullptr;
    size_t ckpt_bytes = 0;
    int ckpt_cap = 0;
    // adjoint work arrays
    double* d_lx = nullptr;
    double* d_lv = nullptr;
    double* d_g = nullptr;
    double* d_theta = nullptr;
    double* d_wts = nullptr;
    double* d_partg = nullptr;
    float4* d_u = nullptr;
    char* d_tape = nullptr;
    size_t tape_step_bytes = 0;
    int tape_cap = 0;
    double* d_parth = nullptr;
    double* d_hist = nullptr;
    int hist_cap = 0;
    std::string err;
};

namespace {

md_status fail(md_box* b, md_status s, const std::string& msg)
{
    if (b) b->err = msg;
    return s;
}

md_status cuda_fail(md_box* b, cudaError_t e, const char* what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return fail(b, MD_ERR_CUDA, buf);
}

#define CK(b, x)                                               \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) return cuda_fail((b), e_, #x);  \
    } while (0)

#define CKS(x)                                  \
    do {                                        \
        md_status s_ = (x);                     \
        if (s_ != MD_OK) return s_;             \
    } while (0)

void* raw_alloc(md_box* b, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (b->alloc) {
        p = b->alloc(bytes, b->actx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void raw_free(md_box* b, void* p)
{
    if (!p) return;
    if (b->free_) b->free_(p, b->actx);
    else cudaFree(p);
}

template <class T>
md_status dev_alloc(md_box* b, T** out, size_t count, bool zero = true)
{
    size_t bytes = sizeof(T) * (count ? count : 1);
    void* p = raw_alloc(b, bytes);
    if (!p) return fail(b, MD_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    b->allocs.push_back({p, bytes});
    if (zero) CK(b, cudaMemsetAsync(p, 0, bytes, b->stream));
    *out = static_cast<T*>(p);
    return MD_OK;
}

void dev_release(md_box* b, void* p)
{
    if (!p) return;
    cudaStreamSynchronize(b->stream);   // no queued work may still use it
    for (size_t i = 0; i < b->allocs.size(); ++i)
        if (b->allocs[i].p == p) {
            raw_free(b, p);
            b->allocs.erase(b->allocs.begin() + (long)i);
            return;
        }
}

md_status ensure_stage(md_box* b, size_t bytes)
{
    if (b->stage_bytes >= bytes) return MD_OK;
    dev_release(b, b->d_stage);
    b->d_stage = nullptr;
    b->stage_bytes = 0;
    char* p;
    CKS(dev_alloc(b, &p, bytes, false));
    b->d_stage = p;
    b->stage_bytes = bytes;
    return MD_OK;
}

void invalidate_graphs(md_box* b)
{
    for (auto& g : b->graphs) {
        cudaGraphExecDestroy(g.exec);
        for (auto e : g.ev) cudaEventDestroy(e);
    }
    b->graphs.clear();
}

Launch lch(md_box* b) { return Launch{std::max(1, std::min((int)b->d.nchunk, b->nsm * 12)), LJ_CHUNK, b->stream}; }
Launch lthermo(md_box* b) { return Launch{std::max(1, std::min(b->d.ntitem, b->nsm * 8)), LJ_THERMO_THREADS, b->stream}; }
Launch lcell(md_box* b) { return Launch{std::max(1, std::min((b->d.ncell + 7) / 8, b->nsm * 8)), 256, b->stream}; }
// The FP32 list-form force kernel and the layout of its (E_pot, W) shares:
// the chunk kernel unless the tiled one is asked for (or chosen by
// md_autotune).  The FP32 list
// kernels leave one double-single share per warp and chunk (chunk kernel)
// or brick (tiled kernel, LJ_BRICK_WARPS = LJ_FORCE_WARPS), the FP64 one an
// FP64 share per warp and chunk, the all-pairs kernels one per chunk.
void apply_force_kernel(md_box* b)
{
    const bool list32 = !b->all_pairs && b->prec != MD_PREC_FP64;
    const bool tiles = list32 && b->force_kernel == MD_FORCE_TILES;
    b->d.force_tiles = tiles ? 1 : 0;
    b->d.pf_stride = b->all_pairs ? 1 : b->prec == MD_PREC_FP64 ? LJ_F64_WARPS : LJ_FORCE_WARPS;
    b->d.pf_ds = list32 ? 1 : 0;
}

Launch lforce(md_box* b)
{
    if (b->d.force_tiles)   // persistent: the resident blocks, bricks handed out in a grid stride
        return Launch{std::max(1, std::min((int)b->d.nbrick, b->nsm * force_tile_blocks_per_sm(b->d.nt == 1))), 0,
                      b->stream};
    int per_sm = b->force_per_sm > 0 ? b->force_per_sm : (b->prec == 2 ? 12 : 6);
    const int items = b->all_pairs ? b->d.nchunk * std::max(1, b->d.ap_js) : b->d.nchunk;
    return Launch{std::max(1, std::min(items, b->nsm * per_sm)), 0, b->stream};
}
Launch llist(md_box* b)
{
    int per_sm = b->list_per_sm > 0 ? b->list_per_sm : 6;
    return Launch{std::max(1, std::min(b->d.nseg, b->nsm * per_sm)), LJ_LIST_THREADS, b->stream};
}

// The lane-per-particle list kernel runs unless the quad kernel is asked for
// (its shared memory does not depend on the capacity).
bool lanes_list(md_box* b)
{
    return b->list_kernel != MD_LIST_QUADS;
}

cudaError_t launch_list(md_box* b, cudaStream_t s)
{
    if (lanes_list(b)) {
        const int per_sm = b->list_per_sm > 0 ? b->list_per_sm : 8;   // resident blocks (64 registers, 19.5 KB)
        const int warps = LJ_LANE_THREADS / 32;
        return launch_nlist_lanes(
            b->d, Launch{std::max(1, std::min((b->d.ncell + warps - 1) / warps, b->nsm * per_sm)), LJ_LANE_THREADS, s});
    }
    Launch l = llist(b);
    l.s = s;
    return launch_nlist(b->d, l);
}

// Fence: internal stream waits for the caller's stream.
md_status enter(md_box* b)
{
    CK(b, cudaSetDevice(b->device));
    CK(b, cudaEventRecord(b->ev, b->ustream));
    CK(b, cudaStreamWaitEvent(b->stream, b->ev, 0));
    return MD_OK;
}

// Finish: wait for the box's work; the caller's stream is ordered after it.
md_status leave(md_box* b)
{
    CK(b, cudaEventRecord(b->ev, b->stream));
    CK(b, cudaStreamWaitEvent(b->ustream, b->ev, 0));
    CK(b, cudaStreamSynchronize(b->stream));
    return MD_OK;
}

// Copy n bytes of input into device memory: returns a device pointer.
md_status input_ptr(md_box* b, const void* src, size_t bytes, const void** dev, size_t stage_off)
{
    if (!src) {
        *dev = nullptr;
        return MD_OK;
    }
    if (is_device_ptr(src)) {
        *dev = src;
        return MD_OK;
    }
    CKS(ensure_stage(b, stage_off + bytes));
    char* dst = static_cast<char*>(b->d_stage) + stage_off;
    CK(b, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream));
    *dev = dst;
    return MD_OK;
}

md_status read_err(md_box* b, int* err2)
{
    CK(b, cudaMemcpyAsync(err2, b->d.err, 3 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));
    return MD_OK;
}

md_status clear_err(md_box* b)
{
    CK(b, cudaMemsetAsync(b->d.err, 0, 3 * sizeof(int), b->stream));
    return MD_OK;
}

// ------------------------------------------------------------------------
// Rebuild / force sequences
// ------------------------------------------------------------------------
// Kernels of one rebuild sequence (bin, scan x2, scatter, rank, gather,
// list; all pairs: binning only re-wraps and re-centres).
int rebuild_kernels(md_box* b) { return b->all_pairs ? 6 : 8; }

md_status enqueue_rebuild(md_box* b, int from_abs, cudaStream_t s = nullptr)
{
    if (!s) s = b->stream;
    auto on = [s](Launch l) {
        l.s = s;
        return l;
    };
    Launch l = on(lch(b));
    CK(b, launch_list_work(b->d, s));   // the cells and chunks the rebuild kernels visit
    CK(b, launch_bin(b->d, from_abs, l));
    Launch lt{std::max(1, std::min((int)b->tiles.size(), b->nsm * 2)), 1024, s};
    CK(b, launch_scan_tiles(b->d, b->d_tiles, (int)b->tiles.size(), b->d_tile_sum, lt));
    CK(b, launch_scatter(b->d, l));
    CK(b, launch_sortgather(b->d, on(b->all_pairs ? lch(b) : lcell(b)), l));
    if (!b->all_pairs) CK(b, launch_list(b, s));
    b->launches += rebuild_kernels(b);
    return MD_OK;
}

// The list update of one step inside a captured step graph: a one-thread
// kernel sets the condition of an IF node from the box-wide rebuild word,
// and the node's body (captured on the box's second stream) holds the
// rebuild sequence, so a step without a build launches one tiny kernel
// instead of the whole sequence (whose kernels exit early anyway).  The
// body's kernels are counted when they run (k_set_rebuild_cond counts the
// true conditions in cond_runs).  Outside a capture, or if the graph API
// refuses the node, the plain sequence is enqueued.
md_status enqueue_rebuild_step(md_box* b)
{
    if (!b->use_cond) return enqueue_rebuild(b, 0);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    CK(b, cudaStreamGetCaptureInfo(b->stream, &cs, nullptr, &g, &deps, &edata, &nd));
    if (cs != cudaStreamCaptureStatusActive) return enqueue_rebuild(b, 0);
    cudaGraphConditionalHandle h;
    CK(b, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    CK(b, launch_set_rebuild_cond(h, b->d, b->d_cond_runs, b->stream));
    b->launches += 1;
    CK(b, cudaStreamGetCaptureInfo(b->stream, &cs, nullptr, &g, &deps, &edata, &nd));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(b, cudaGraphAddNode(&node, g, deps, edata, nd, &p));
    CK(b, cudaStreamUpdateCaptureDependencies(b->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    CK(b, cudaStreamBeginCaptureToGraph(b->cstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = b->launches;
    md_status st = enqueue_rebuild(b, 0, b->cstream);
    b->launches = l0;   // counted per execution instead
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cstream, &out);
    if (st != MD_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(b, ce, "cudaStreamEndCapture (rebuild body)");
    return MD_OK;
}

md_status enqueue_force(md_box* b, int energy, double* thermo_out_dev)
{
    CK(b, launch_force(b->d, energy, lforce(b)));
    b->launches += 1;
    if (energy && thermo_out_dev) {
        CK(b, launch_thermo(b->d, thermo_out_dev, 0, lthermo(b)));
        b->launches += 1;
    }
    return MD_OK;
}

md_status set_all_rebuild(md_box* b)
{
    std::vector<int> ones(b->nrep, 1);
    CK(b, cudaMemcpyAsync(b->d.rebuild_req, ones.data(), sizeof(int) * b->nrep,
                          cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaMemcpyAsync(b->d.any_req, ones.data(), sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));   // `ones` is pageable and local
    return MD_OK;
}

md_status alloc_lists(md_box* b, int K)
{
    K = round_up(K, LJ_ROW_BLOCK);   // the FP32 force kernel reads rows in whole blocks
    if (b->d.nbr) dev_release(b, b->d.nbr);
    b->d.nbr = nullptr;
    b->d.K = K;
    uint32_t* nb;
    CKS(dev_alloc(b, &nb, (size_t)b->np * (size_t)K + 64, false));
    b->d.nbr = nb;
    invalidate_graphs(b);
    return MD_OK;
}

// Segments: runs of S cells along x inside each cell row.  S is chosen so
// that a tile (9 rows x (S + 2) cells) holds ~1400 particles on average,
// well inside the 2048 a 16-bit list entry can address.
md_status make_segments(md_box* b, bool shrink)
{
    b->segs.clear();
    for (int r = 0; r < b->nrep; ++r) {
        RepDev& R = b->reps[r];
        if (shrink) {
            R.S = std::max(1, R.S / 2);
        } else if (b->seg_cells > 0) {
            R.S = std::max(1, std::min(std::min(b->seg_cells, R.nc[0]), LJ_SEG_MAX_CELLS));
        } else {
            double per_cell = R.ncell > 0 ? (double)R.n / R.ncell : 0.0;
            int S = per_cell > 0 ? (int)std::floor(1400.0 / (9.0 * per_cell)) - 2 : R.nc[0];
            R.S = std::max(1, std::min(std::min(S, R.nc[0]), LJ_SEG_MAX_CELLS));
        }
        R.seg_off = (int)b->segs.size();
        for (int row = 0; row < R.nc[1] * R.nc[2]; ++row)
            for (int x0 = 0; x0 < R.nc[0]; x0 += R.S)
                b->segs.push_back(make_int4(r, x0, row, std::min(R.S, R.nc[0] - x0)));
        R.nseg = (int)b->segs.size() - R.seg_off;
    }
    BoxDev& d = b->d;
    d.nseg = (int)b->segs.size();
    invalidate_graphs(b);
    dev_release(b, b->d_seg);
    CKS(dev_alloc(b, &b->d_seg, b->segs.size(), false));
    d.seg = b->d_seg;
    CK(b, cudaMemcpyAsync(b->d_seg, b->segs.data(), sizeof(int4) * b->segs.size(),
                          cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaMemcpyAsync(b->d_rep, b->reps.data(), sizeof(RepDev) * b->reps.size(),
                          cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));
    return MD_OK;
}

// The cell grid of every replica (particle binning, Sec. 3): floor(L / (rl *
// cell_scale)) cells per dimension (cell_scale >= 1: every cell edge is at
// least the list radius, as the 27-cell stencil needs), scan tiles, segments
// and a list capacity for the densest replica.  The caller re-bins (full
// rebuild) afterwards.
md_status make_grid(md_box* b)
{
    BoxDev& d = b->d;
    invalidate_graphs(b);
    b->tiles.clear();
    b->bricks.clear();
    int cell_off = 0;
    double maxdens = 0.0;
    for (int r = 0; r < b->nrep; ++r) {
        RepDev& R = b->reps[r];
        for (int c = 0; c < 3; ++c) {
            R.nc[c] = std::max(1, (int)std::floor(R.L[c] / (b->rl * b->cell_scale)));
            R.ell[c] = R.L[c] / R.nc[c];
            R.inv_ell[c] = (double)R.nc[c] / R.L[c];
            R.ellf[c] = (float)R.ell[c];
            R.ell_lo[c] = (float)(R.ell[c] - (double)R.ellf[c]);
        }
        R.cell_off = cell_off;
        R.ncell = R.nc[0] * R.nc[1] * R.nc[2];
        // bricks of the tiled force kernel: 2 cells along an axis where the
        // brick-centre frame keeps tile coordinates below 8 (2 ell + drift),
        // else 1; x fastest, so that neighbouring blocks share tile cells in L2
        for (int c = 0; c < 3; ++c) R.br[c] = (R.nc[c] >= 2 && R.ellf[c] < 3.9f) ? 2 : 1;
        R.brick_off = (int)b->bricks.size();
        for (int z = 0; z < R.nc[2]; z += R.br[2])
            for (int y = 0; y < R.nc[1]; y += R.br[1])
                for (int x = 0; x < R.nc[0]; x += R.br[0]) b->bricks.push_back(make_int4(r, x, y, z));
        R.nbrick = (int)b->bricks.size() - R.brick_off;
        int first_tile = (int)b->tiles.size();
        for (int c0 = 0; c0 < R.ncell; c0 += ljmd_scan_tile_cells())
            b->tiles.push_back(make_int4(r, cell_off + c0,
                                         cell_off + std::min(R.ncell, c0 + ljmd_scan_tile_cells()),
                                         first_tile));
        cell_off += R.ncell;
        maxdens = std::max(maxdens, R.n / (R.L[0] * R.L[1] * R.L[2]));
    }
    d.ncell = cell_off;
    d.ell1 = make_float3(b->reps[0].ellf[0], b->reps[0].ellf[1], b->reps[0].ellf[2]);
    CK(b, cudaMemcpyAsync(b->d_rep, b->reps.data(), sizeof(RepDev) * b->reps.size(),
                          cudaMemcpyHostToDevice, b->stream));
    dev_release(b, d.cell_count);
    dev_release(b, d.cell_start);
    dev_release(b, d.cell_end);
    dev_release(b, (void*)d.cell_rep);
    dev_release(b, b->d_tiles);
    dev_release(b, b->d_brick);
    b->d_brick = nullptr;
    dev_release(b, b->d_tile_sum);
    d.cell_count = d.cell_start = d.cell_end = nullptr;
    d.cell_rep = nullptr;
    CKS(dev_alloc(b, &d.cell_count, d.ncell));
    CKS(dev_alloc(b, &d.cell_start, d.ncell));
    CKS(dev_alloc(b, &d.cell_end, d.ncell));
    int* cr;
    CKS(dev_alloc(b, &cr, d.ncell, false));
    {
        std::vector<int> hc(d.ncell);
        for (int r = 0; r < b->nrep; ++r)
            for (int c = 0; c < b->reps[r].ncell; ++c) hc[b->reps[r].cell_off + c] = r;
        CK(b, cudaMemcpyAsync(cr, hc.data(), sizeof(int) * d.ncell, cudaMemcpyHostToDevice, b->stream));
        CK(b, cudaStreamSynchronize(b->stream));
    }
    d.cell_rep = cr;
    CKS(dev_alloc(b, &b->d_tiles, b->tiles.size(), false));
    CKS(dev_alloc(b, &b->d_tile_sum, b->tiles.size()));
    CK(b, cudaMemcpyAsync(b->d_tiles, b->tiles.data(), sizeof(int4) * b->tiles.size(),
                          cudaMemcpyHostToDevice, b->stream));
    CKS(dev_alloc(b, &b->d_brick, b->bricks.size(), false));
    CK(b, cudaMemcpyAsync(b->d_brick, b->bricks.data(), sizeof(int4) * b->bricks.size(),
                          cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));   // `bricks` may change before the copy would run
    d.brick = b->d_brick;
    d.nbrick = (int)b->bricks.size();
    {   // (E_pot, W) shares: 8 per chunk or per brick
        const size_t need = 2 * LJ_FORCE_WARPS * std::max<size_t>(1, std::max(b->chunks.size(), b->bricks.size()));
        if (need > b->pf_cap) {
            dev_release(b, d.part_f);
            d.part_f = nullptr;
            b->pf_cap = 0;
            CKS(dev_alloc(b, &d.part_f, need));
            b->pf_cap = need;
        }
    }
    CKS(make_segments(b, false));
    // list capacity: expected neighbours at the densest replica, +30 %
    double expect = b->all_pairs ? 0.0 : maxdens * 4.18879020478639 * b->rl * b->rl * b->rl;
    int K = round_up((int64_t)(1.3 * expect) + 16, 8);   // all pairs: no lists, a token row
    if (b->min_capacity > 0) K = round_up(b->min_capacity, 8);
    CKS(alloc_lists(b, K));
    b->autofit = true;
    return MD_OK;
}

// Rebuild all replicas now (forced), regrowing the lists until they fit,
// then recompute the forces.
md_status full_rebuild(md_box* b)
{
    for (int attempt = 0; attempt < 24; ++attempt) {
        CKS(clear_err(b));
        CKS(set_all_rebuild(b));
        CKS(enqueue_rebuild(b, b->fresh_abs ? 1 : 0));
        int e2[3];
        CKS(read_err(b, e2));
        b->binned = true;
        if (e2[0] & LJ_ERRBIT_TIMEOUT) return fail(b, MD_ERR_TIMEOUT, "list build: device wait timed out");
        if (e2[0] & LJ_ERRBIT_TILE) {
            bool can_shrink = false;
            for (const RepDev& R : b->reps) can_shrink = can_shrink || R.S > 1;
            if (!can_shrink)
                return fail(b, MD_ERR_CAPACITY,
                            "list build: the 27 cells around one cell hold more than 2048 particles "
                            "(cells too large for the density)");
            CKS(make_segments(b, true));
            continue;
        }
        if (e2[0] & LJ_ERRBIT_CAPACITY) {
            // binning and sorting completed (xabs still holds the exact
            // positions, now in sorted slots); only the lists were cut short
            int K = round_up((int64_t)(e2[1] * 1.15) + 8, 8);
            CKS(alloc_lists(b, K));
            continue;
        }
        b->fresh_abs = true;
        // automatic capacity: fit it to the longest list (+10 % and 8) so
        // the padded rows the force kernel streams stay short
        if (b->min_capacity == 0 && b->autofit) {
            int Kfit = round_up((int64_t)(e2[2] * 1.1) + 8, 8);
            b->autofit = false;
            if (Kfit + 8 < b->d.K) {
                CKS(alloc_lists(b, Kfit));
                continue;
            }
        }
        CKS(enqueue_force(b, 0, nullptr));
        return MD_OK;
    }
    return fail(b, MD_ERR_CAPACITY, "neighbour list kept overflowing");
}

// Apply a cell layout (cell scale, order inside cells): a new cell grid
// when the scale changes (positions first put back into xabs), then a full
// rebuild in the new order.  The box's positions are unchanged.
static md_status apply_layout(md_box* b, double scale, int order)
{
    b->order = order;
    b->d.order = order;
    invalidate_graphs(b);
    if (scale != b->cell_scale) {
        b->cell_scale = scale;
        if (!b->fresh_abs) {
            CK(b, launch_materialize(b->d, lch(b)));
            b->fresh_abs = true;
        }
        CKS(make_grid(b));
    }
    b->rec_valid = false;
    return full_rebuild(b);
}

// A layout whose lists cannot be built (a 27-cell tile over 2048 particles)
// is refused: the previous layout is put back and its lists rebuilt, and the
// refusal's status and message are returned.
md_status set_layout(md_box* b, double scale, int order)
{
    if (scale == b->cell_scale && order == b->order) return MD_OK;
    const double old_scale = b->cell_scale;
    const int old_order = b->order;
    const md_status st = apply_layout(b, scale, order);
    if (st == MD_OK || st != MD_ERR_CAPACITY) return st;
    const std::string why = b->err;
    CKS(clear_err(b));
    CKS(apply_layout(b, old_scale, old_order));
    return fail(b, st, why);
}

md_status snapshot_setup(md_box* b)
{
    int np = b->np;
    b->snap_src.clear();
    size_t accb = sizeof(double) * 3 * (size_t)np;
    b->snap_src.push_back({b->d.off, accb});
    b->snap_src.push_back({b->d.vel, accb});
    b->snap_src.push_back({b->d.img, sizeof(int) * 3 * (size_t)np});
    b->snap_src.push_back({b->d.uid, sizeof(int) * (size_t)np});
    b->snap_src.push_back({b->d.type, sizeof(int) * (size_t)np});
    b->snap_src.push_back({b->d.cell, sizeof(int) * (size_t)np});
    b->snap_src.push_back({b->d_step_ctr, sizeof(long long)});
    size_t tot = 0;
    for (auto& s : b->snap_src) tot += (s.second + 255) & ~(size_t)255;
    if (b->snap_bytes < tot) {
        dev_release(b, b->d_snap);
        char* p;
        CKS(dev_alloc(b, &p, tot, false));
        b->d_snap = p;
        b->snap_bytes = tot;
    }
    return MD_OK;
}

md_status snapshot(md_box* b, bool restore)
{
    size_t o = 0;
    for (auto& s : b->snap_src) {
        char* dst = static_cast<char*>(b->d_snap) + o;
        if (restore) CK(b, cudaMemcpyAsync(s.first, dst, s.second, cudaMemcpyDeviceToDevice, b->stream));
        else CK(b, cudaMemcpyAsync(dst, s.first, s.second, cudaMemcpyDeviceToDevice, b->stream));
        o += (s.second + 255) & ~(size_t)255;
    }
    return MD_OK;
}

// The velocity-Verlet loop for `n` steps (Sec. 3, Fig. 1): integrate,
// conditional list update, force, finalize (fused with the next integrate).
// With `ge` set, events bracket every phase of every step (profiling).
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Copy the state a Hessian-vector product needs (FP32 offsets, slot -> user
// map, lists) into tape slot m.
md_status tape_save(md_box* b, int m)
{
    const size_t np = (size_t)b->np;
    char* t = b->d_tape + (size_t)m * b->tape_step_bytes;
    CK(b, cudaMemcpyAsync(t, b->d.posq, np * 16, cudaMemcpyDeviceToDevice, b->stream));
    t += al256(np * 16);
    CK(b, cudaMemcpyAsync(t, b->d.uid, np * 4, cudaMemcpyDeviceToDevice, b->stream));
    t += al256(np * 4);
    CK(b, cudaMemcpyAsync(t, b->d.nbr_count, np * 4, cudaMemcpyDeviceToDevice, b->stream));
    t += al256(np * 4);
    CK(b, cudaMemcpyAsync(t, b->d.nbr, np * (size_t)b->d.K * 4, cudaMemcpyDeviceToDevice, b->stream));
    return MD_OK;
}

BoxDev tape_view(md_box* b, int m)
{
    const size_t np = (size_t)b->np;
    BoxDev v = b->d;
    char* t = b->d_tape + (size_t)m * b->tape_step_bytes;
    v.posq = reinterpret_cast<float4*>(t);
    t += al256(np * 16);
    v.uid = reinterpret_cast<int*>(t);
    t += al256(np * 4);
    v.nbr_count = reinterpret_cast<int*>(t);
    t += al256(np * 4);
    v.nbr = reinterpret_cast<uint32_t*>(t);
    return v;
}

md_status enqueue_steps(md_box* b, int64_t n, double dt, int energy, double* ring, GraphEnt* ge,
                        bool tape = false)
{
    Launch l = lch(b);
    // The energy reduction of step s reads the force shares of step s - 1 and
    // the kinetic shares of this integrate: it runs on a branch (side stream)
    // beside the list update and joins before the force kernel rewrites them.
    const Launch lt{lthermo(b).grid, LJ_THERMO_THREADS, b->side};
    size_t rs = (size_t)b->nrep * 4;
    auto mark = [&](int64_t s, int ph, int end, cudaStream_t st) -> cudaError_t {
        if (!ge) return cudaSuccess;
        size_t k = (size_t)(s * 4 + ph);
        ge->used[k] = 1;
        // an external record becomes an event-record node of the graph
        return cudaEventRecordWithFlags(ge->ev[2 * k + end], st, cudaEventRecordExternal);
    };
    bool joined = true;
    auto join = [&]() -> cudaError_t {
        if (joined) return cudaSuccess;
        joined = true;
        return cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    };
    for (int64_t s = 0; s <= n; ++s) {
        int mode = s == 0 ? LJ_STEP_FIRST : (s == n ? LJ_STEP_LAST : LJ_STEP_MID);
        CK(b, mark(s, 0, 0, b->stream));
        CK(b, launch_integrate(b->d, mode, s == 0 ? 0 : energy, dt, (int)(s > 0 ? s - 1 : 0), l));
        CK(b, mark(s, 0, 1, b->stream));
        b->launches += 1;
        if (s > 0 && energy) {
            CK(b, cudaEventRecord(b->ev_fork, b->stream));
            CK(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0));
            CK(b, mark(s, 3, 0, b->side));
            CK(b, launch_thermo(b->d, ring + (s - 1) * rs, 1, lt));
            CK(b, mark(s, 3, 1, b->side));
            CK(b, cudaEventRecord(b->ev_join, b->side));
            joined = false;
            b->launches += 1;
        }
        if (s == n) break;
        CK(b, mark(s, 1, 0, b->stream));
        if (!b->all_pairs) CKS(enqueue_rebuild_step(b));   // all pairs: the drift keeps offsets wrapped
        CK(b, mark(s, 1, 1, b->stream));
        CK(b, join());
        CK(b, mark(s, 2, 0, b->stream));
        CK(b, launch_force(b->d, energy, lforce(b)));
        CK(b, mark(s, 2, 1, b->stream));
        b->launches += 1;
        if (tape) CKS(tape_save(b, (int)s + 1));
    }
    CK(b, join());
    // steps since md_set_thermostat (the thermostat's counter), on the device
    if (!tape) {
        CK(b, launch_step_advance(b->d.step_ctr, n, b->stream));
        b->launches += 1;
    }
    return MD_OK;
}

// ------------------------------------------------------------------------
// Checkpoints of a recorded run.  A checkpoint is taken right after a forced
// list build, so restoring it and rebuilding only the lists (k_nlist from the
// saved offsets, cell ranges and build positions) reproduces the recorded
// state bit for bit.
// ------------------------------------------------------------------------
md_status ckpt_setup(md_box* b, int C)
{
    const size_t np = (size_t)b->np, nc = (size_t)b->d.ncell;
    b->ck_src.clear();
    b->ck_src.push_back({b->d.off, 24 * np});
    b->ck_src.push_back({b->d.vel, 24 * np});
    b->ck_src.push_back({b->d.img, 12 * np});
    b->ck_src.push_back({b->d.uid, 4 * np});
    b->ck_src.push_back({b->d.type, 4 * np});
    b->ck_src.push_back({b->d.cell, 4 * np});
    b->ck_src.push_back({b->d.posq, 16 * np});
    b->ck_src.push_back({b->d.ref, 16 * np});
    b->ck_src.push_back({b->d.xabs, 24 * np});
    b->ck_src.push_back({b->d.cell_start, 4 * nc});
    b->ck_src.push_back({b->d.cell_end, 4 * nc});
    size_t per = 0;
    for (auto& a : b->ck_src) per += al256(a.second);
    if (b->ckpt_bytes != per || b->ckpt_cap < C) {
        dev_release(b, b->d_ckpt);
        b->d_ckpt = nullptr;
        CKS(dev_alloc(b, &b->d_ckpt, per * (size_t)C, false));
        b->ckpt_bytes = per;
        b->ckpt_cap = C;
    }
    return MD_OK;
}

md_status ckpt_copy(md_box* b, int c, bool restore)
{
    char* base = b->d_ckpt + (size_t)c * b->ckpt_bytes;
    for (auto& a : b->ck_src) {
        if (restore) CK(b, cudaMemcpyAsync(a.first, base, a.second, cudaMemcpyDeviceToDevice, b->stream));
        else CK(b, cudaMemcpyAsync(base, a.first, a.second, cudaMemcpyDeviceToDevice, b->stream));
        base += al256(a.second);
    }
    return MD_OK;
}

// Lists from the restored build state, then the forces (no re-binning).
md_status replay_lists(md_box* b)
{
    CKS(set_all_rebuild(b));
    CK(b, launch_list_work(b->d, b->stream));
    CK(b, launch_list(b, b->stream));
    CK(b, launch_force(b->d, 0, lforce(b)));
    b->launches += 3;
    return MD_OK;
}

md_status get_graph(md_box* b, int64_t n, double dt, int energy, cudaGraphExec_t* out)
{
    for (auto& g : b->graphs)
        if (g.nsteps == n && g.dt == dt && g.energy == energy) {
            *out = g.exec;
            return MD_OK;
        }
    if (b->graphs.size() >= 8) invalidate_graphs(b);
    GraphEnt ge{n, dt, energy, nullptr, 0, {}, {}};
    if (b->profiling) {
        ge.ev.resize((size_t)(n + 1) * 8);
        ge.used.assign((size_t)(n + 1) * 4, 0);
        for (auto& e : ge.ev) CK(b, cudaEventCreate(&e));
    }
    // with conditional list-update nodes first; should the runtime refuse
    // them, once more with the plain (early-exit) rebuild sequence
    for (;;) {
        cudaGraph_t graph = nullptr;
        int64_t l0 = b->launches;
        CK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        md_status st = enqueue_steps(b, n, dt, energy, b->d_thermo, b->profiling ? &ge : nullptr);
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        ge.kernels = b->launches - l0;
        b->launches = l0;
        if (st == MD_OK && ce == cudaSuccess) {
            ce = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            graph = nullptr;
            if (ce == cudaSuccess) break;
        }
        if (graph) cudaGraphDestroy(graph);
        if (!b->use_cond) {
            if (st != MD_OK) return st;
            return cuda_fail(b, ce, "step graph capture");
        }
        cudaGetLastError();
        b->use_cond = false;
    }
    b->graphs.push_back(ge);
    *out = ge.exec;
    return MD_OK;
}

md_status ensure_thermo(md_box* b, int64_t steps)
{
    int64_t need = steps * b->nrep * 4;
    if (b->thermo_cap >= need) return MD_OK;
    invalidate_graphs(b);   // graphs hold the ring pointer
    dev_release(b, b->d_thermo);
    b->d_thermo = nullptr;
    CKS(dev_alloc(b, &b->d_thermo, (size_t)need));
    b->thermo_cap = need;
    return MD_OK;
}

void copy_reps_to(md_box* b, BoxDev& d)
{
    d.nrep = b->nrep;
    d.np = b->np;
    d.nchunk = (int)b->chunks.size();
    d.prec = b->prec;
}

// Time `reps` launches of fn on the box stream (milliseconds per launch).
template <class F>
md_status time_launches(md_box* b, int reps, F fn, float* ms_out)
{
    cudaEvent_t e0, e1;
    CK(b, cudaEventCreate(&e0));
    CK(b, cudaEventCreate(&e1));
    CKS(fn());   // warm-up
    CK(b, cudaEventRecord(e0, b->stream));
    for (int i = 0; i < reps; ++i) CKS(fn());
    CK(b, cudaEventRecord(e1, b->stream));
    CK(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(b, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms / (float)std::max(1, reps);
    return MD_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

md_status md_set_allocator(md_alloc_fn alloc, md_free_fn free_, void* ctx)
{
    if ((alloc == nullptr) != (free_ == nullptr)) return MD_ERR_ARG;
    g_alloc = alloc;
    g_free = free_;
    g_ctx = ctx;
    return MD_OK;
}

const char* md_status_string(md_status s)
{
    switch (s) {
    case MD_OK: return "ok";
    case MD_ERR_ARG: return "invalid argument";
    case MD_ERR_CUDA: return "CUDA error";
    case MD_ERR_OOM: return "out of device memory";
    case MD_ERR_CAPACITY: return "neighbour list capacity exceeded";
    case MD_ERR_BOX_TOO_SMALL: return "list radius not below half the box";
    case MD_ERR_NONFINITE: return "non-finite force or position";
    case MD_ERR_TIMEOUT: return "device wait timed out";
    case MD_ERR_STATE: return "no recorded forward run";
    }
    return "unknown status";
}

const char* md_last_error(const md_box* b) { return b ? b->err.c_str() : "null box"; }

md_status md_batch_create(md_box** out, int32_t nrep, const int64_t* n, const double* box,
                          const int32_t* type, const double* pos, const double* vel,
                          md_precision prec, void* stream)
{
    if (!out || nrep < 1 || !n || !box || (prec < 0 || prec > 2)) return MD_ERR_ARG;
    *out = nullptr;
    int64_t ntot = 0, np = 0;
    for (int r = 0; r < nrep; ++r) {
        if (n[r] < 0) return MD_ERR_ARG;
        for (int c = 0; c < 3; ++c)
            if (!(box[3 * r + c] > 0.0) || !std::isfinite(box[3 * r + c])) return MD_ERR_ARG;
        ntot += n[r];
        np += round_up(n[r], 32);
    }
    if (ntot > 0 && !pos) return MD_ERR_ARG;
    if (np >= (int64_t(1) << LJ_IDX_BITS)) return MD_ERR_ARG;
    md_box* b = new md_box();
    b->alloc = g_alloc;
    b->free_ = g_free;
    b->actx = g_ctx;
    b->prec = prec;
    b->nrep = nrep;
    b->ntot = ntot;
    b->np = (int)std::max<int64_t>(np, 32);
    b->ustream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (b->ev_join) cudaEventDestroy(b->ev_join);
        if (b->ev_fork) cudaEventDestroy(b->ev_fork);
        if (b->side) cudaStreamDestroy(b->side);
        if (b->ev) cudaEventDestroy(b->ev);
        if (b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return MD_ERR_CUDA;
    }
    // replicas and work items
    int64_t poff = 0, uoff = 0;
    for (int r = 0; r < nrep; ++r) {
        RepDev R{};
        for (int c = 0; c < 3; ++c) {
            R.L[c] = box[3 * r + c];
            R.wrap_hi[c] = R.L[c] * (1.0 - std::ldexp(1.0, -50));
        }
        R.p_off = (int)poff;
        R.n = (int)n[r];
        R.u_off = (int)uoff;
        R.chunk_off = (int)b->chunks.size();
        for (int64_t p = 0; p < n[r]; p += LJ_CHUNK)
            b->chunks.push_back(make_int4(r, (int)(poff + p), (int)(poff + std::min<int64_t>(p + LJ_CHUNK, n[r])),
                                          (int)b->chunks.size()));
        R.nchunk = (int)b->chunks.size() - R.chunk_off;
        R.ti_off = (int)b->titems.size();
        for (int c = 0; c < std::max(1, R.nchunk); c += LJ_THERMO_CHUNKS)
            b->titems.push_back(
                make_int4(r, R.chunk_off + c, R.chunk_off + std::min(c + LJ_THERMO_CHUNKS, R.nchunk), 0));
        R.nti = (int)b->titems.size() - R.ti_off;
        b->reps.push_back(R);
        poff += round_up(n[r], 32);
        uoff += n[r];
    }
    md_status st = [&]() -> md_status {
        BoxDev& d = b->d;
        copy_reps_to(b, d);
        size_t np3 = 3 * (size_t)b->np;
        CKS(dev_alloc(b, &b->d_rep, b->reps.size()));
        CKS(dev_alloc(b, &b->d_chunk, b->chunks.size()));
        int4* ti;
        CKS(dev_alloc(b, &ti, b->titems.size(), false));
        CK(b, cudaMemcpyAsync(ti, b->titems.data(), sizeof(int4) * b->titems.size(), cudaMemcpyHostToDevice,
                              b->stream));
        d.titem = ti;
        d.ntitem = (int)b->titems.size();
        CKS(dev_alloc(b, &d.part_t, 3 * b->titems.size()));
        CKS(dev_alloc(b, &d.tcount, nrep));
        CKS(dev_alloc(b, &b->d_lj, 1));
        CK(b, cudaMemcpyAsync(b->d_chunk, b->chunks.data(), sizeof(int4) * b->chunks.size(),
                              cudaMemcpyHostToDevice, b->stream));
        d.rep = b->d_rep;
        d.chunk = b->d_chunk;
        d.lj = b->d_lj;
        CKS(dev_alloc(b, &d.posq, (size_t)b->np + 1));
        static const float4 sentinel = {LJ_SENTINEL_OFF, LJ_SENTINEL_OFF, LJ_SENTINEL_OFF, 0.f};   // species 0
        CK(b, cudaMemcpyAsync(d.posq + b->np, &sentinel, sizeof(float4), cudaMemcpyHostToDevice, b->stream));
        CKS(dev_alloc(b, &d.ref, b->np));
        CKS(dev_alloc(b, &d.off, np3));
        CKS(dev_alloc(b, &d.vel, np3));
        CKS(dev_alloc(b, &d.img, np3));
        CKS(dev_alloc(b, &d.uid, b->np));
        CKS(dev_alloc(b, &d.type, b->np));
        CKS(dev_alloc(b, &d.cell, b->np));
        CKS(dev_alloc(b, &d.xabs, np3));
        if (prec == MD_PREC_FP64) CKS(dev_alloc(b, &d.force64, np3));
        else CKS(dev_alloc(b, &d.force4, b->np));
        CKS(dev_alloc(b, &d.xabsB, np3));
        CKS(dev_alloc(b, &d.offB, np3));
        CKS(dev_alloc(b, &d.velB, np3));
        CKS(dev_alloc(b, &d.imgB, np3));
        CKS(dev_alloc(b, &d.uidB, b->np));
        CKS(dev_alloc(b, &d.typeB, b->np));
        CKS(dev_alloc(b, &d.cellB, b->np));
        CKS(dev_alloc(b, &d.perm, b->np));
        CKS(dev_alloc(b, &d.dst, b->np));
        CKS(dev_alloc(b, &d.nbr_count, b->np));
        CKS(dev_alloc(b, &d.disp_max, nrep));
        CKS(dev_alloc(b, &d.rebuild_req, nrep));
        CKS(dev_alloc(b, &d.any_req, 1));
        CKS(dev_alloc(b, &b->d_step_ctr, 1));
        d.step_ctr = b->d_step_ctr;
        CKS(dev_alloc(b, &b->d_tstat_T, nrep));
        d.tstat_T = b->d_tstat_T;
        d.tstat_thr = 0u;
        CKS(dev_alloc(b, &d.nbuild, nrep));
        {
            int* lw;
            CKS(dev_alloc(b, &lw, 1 + 3 * (size_t)nrep + 2));
            d.lw_hdr = lw;
            d.lw_rep = lw + 1;
            d.lw_off = lw + 1 + nrep;
            d.lw_coff = lw + 2 + 2 * nrep;
        }
        CKS(dev_alloc(b, &d.err, 4));
        CKS(dev_alloc(b, &b->d_cond_runs, 1));
        CKS(dev_alloc(b, &d.part_k, LJ_KIN_WARPS * std::max<size_t>(1, b->chunks.size())));
        // (E_pot, W) shares, 8 per chunk (chunk kernel) or brick (tiled
        // kernel; make_grid grows the array with the bricks)
        b->pf_cap = 2 * LJ_FORCE_WARPS * std::max<size_t>(1, b->chunks.size());
        CKS(dev_alloc(b, &d.part_f, b->pf_cap));
        apply_force_kernel(b);
        CKS(dev_alloc(b, &b->d_type_user, std::max<int64_t>(1, ntot)));
        CK(b, cudaMemcpyAsync(b->d_rep, b->reps.data(), sizeof(RepDev) * b->reps.size(),
                              cudaMemcpyHostToDevice, b->stream));
        CKS(enter(b));
        if (ntot > 0) {
            const void *dpos, *dvel = nullptr, *dtype = nullptr;
            size_t pb = sizeof(double) * 3 * (size_t)ntot;
            CKS(ensure_stage(b, 2 * pb + sizeof(int) * (size_t)ntot + 256));
            CKS(input_ptr(b, pos, pb, &dpos, 0));
            CKS(input_ptr(b, vel, pb, &dvel, pb));
            CKS(input_ptr(b, type, sizeof(int) * (size_t)ntot, &dtype, 2 * pb));
            if (dtype) {
                CK(b, cudaMemcpyAsync(b->d_type_user, dtype, sizeof(int) * (size_t)ntot,
                                      cudaMemcpyDeviceToDevice, b->stream));
            }
            CK(b, launch_upload(d, static_cast<const double*>(dpos), static_cast<const double*>(dvel),
                                b->d_type_user, 1, lch(b)));
        }
        CKS(snapshot_setup(b));
        CKS(leave(b));
        return MD_OK;
    }();
    if (st != MD_OK) {
        md_box_destroy(b);
        return st;
    }
    *out = b;
    return MD_OK;
}

md_status md_box_create(md_box** out, int64_t n, const double box[3], const int32_t* type,
                        const double* pos, const double* vel, md_precision prec, void* stream)
{
    return md_batch_create(out, 1, &n, box, type, pos, vel, prec, stream);
}

md_status md_box_destroy(md_box* b)
{
    if (!b) return MD_ERR_ARG;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    invalidate_graphs(b);
    for (auto& a : b->allocs) raw_free(b, a.p);
    b->allocs.clear();
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->cstream) cudaStreamDestroy(b->cstream);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return MD_OK;
}

md_status md_set_lj(md_box* b, int32_t ntypes, const double* eps, const double* sigma,
                    const double* rcut, double skin, int32_t energy_shift)
{
    if (!b || ntypes < 1 || ntypes > LJ_MAXT || !eps || !sigma || !rcut || !(skin >= 0.0))
        return fail(b, MD_ERR_ARG, "md_set_lj: bad arguments");
    int nt = ntypes;
    double rcmax = 0.0;
    int ninf = 0;
    for (int a = 0; a < nt; ++a)
        for (int c = 0; c < nt; ++c) {
            int k = a * nt + c, t = c * nt + a;
            if (!(eps[k] > 0) || !(sigma[k] > 0) || !(rcut[k] > 0) || eps[k] != eps[t] ||
                sigma[k] != sigma[t] || rcut[k] != rcut[t] || std::isnan(rcut[k]))
                return fail(b, MD_ERR_ARG, "md_set_lj: parameters must be positive and symmetric");
            rcmax = std::max(rcmax, rcut[k]);
            ninf += std::isinf(rcut[k]) ? 1 : 0;
        }
    if (ninf != 0 && ninf != nt * nt)
        return fail(b, MD_ERR_ARG, "md_set_lj: cutoffs must be all finite or all infinite (all pairs)");
    const bool all_pairs = ninf != 0;
    double rl = rcmax + skin;
    for (int r = 0; r < b->nrep; ++r)
        for (int c = 0; c < 3; ++c)
            if (!all_pairs && !(rl < 0.5 * b->reps[r].L[c]))
                return fail(b, MD_ERR_BOX_TOO_SMALL, "md_set_lj: rc + skin >= L/2");
    CKS(enter(b));
    // types given at creation must be < ntypes: checked on the host copy
    if (b->ntot > 0) {
        std::vector<int> t(b->ntot);
        CK(b, cudaMemcpyAsync(t.data(), b->d_type_user, sizeof(int) * b->ntot, cudaMemcpyDeviceToHost,
                              b->stream));
        CK(b, cudaStreamSynchronize(b->stream));
        for (int v : t)
            if (v < 0 || v >= nt) return fail(b, MD_ERR_ARG, "md_set_lj: particle type out of range");
    }
    // new cell grid: if it changes while particles are binned, put positions
    // back into xabs first
    bool grid_changes = !b->lj_set || rl != b->rl || all_pairs != b->all_pairs;
    b->all_pairs = all_pairs;
    b->d.all_pairs = all_pairs ? 1 : 0;
    apply_force_kernel(b);   // the force kernel and its (E_pot, W) shares
    if (all_pairs && !b->d.ap_cnt) {
        // j slices per chunk: enough work items to fill the GPU, each slice
        // at least ~128 particles
        int nmax = 1;
        for (auto& R : b->reps) nmax = std::max(nmax, R.n);
        const int nch = std::max(1, (int)b->chunks.size());
        const int js = std::max(1, std::min((b->nsm * 4 + nch - 1) / nch, std::max(1, nmax / 128)));
        b->d.ap_js = js;
        CKS(dev_alloc(b, &b->d.ap_part, (size_t)js * b->np, false));
        if (b->prec == MD_PREC_FP64) CKS(dev_alloc(b, &b->d.ap_part64, (size_t)js * 3 * b->np, false));
        CKS(dev_alloc(b, &b->d.ap_pe, 2 * (size_t)js * nch, false));
        CKS(dev_alloc(b, &b->d.ap_cnt, nch));
    }
    if (b->lj_set && grid_changes && !b->fresh_abs) {
        CK(b, launch_materialize(b->d, lch(b)));
        b->fresh_abs = true;
    }
    LJDev h{};
    h.nt = nt;
    h.shift_on = energy_shift ? 1 : 0;
    for (int k = 0; k < nt * nt; ++k) {
        double s2 = sigma[k] * sigma[k];
        double rc2 = rcut[k] * rcut[k];
        double c6 = (s2 / rc2) * (s2 / rc2) * (s2 / rc2);
        double sh = energy_shift ? 4.0 * eps[k] * (c6 * c6 - c6) : 0.0;
        double s6 = s2 * s2 * s2;
        double sg = sigma[k];
        h.a12[k] = (float)(672.0 * eps[k] * s6 * s6);
        h.a6[k] = (float)(192.0 * eps[k] * s6);
        h.g12[k] = (float)(576.0 * eps[k] * s6 * s6 / sg);
        h.g6[k] = (float)(144.0 * eps[k] * s6 / sg);
        h.inv_eps[k] = (float)(1.0 / eps[k]);
        h.c12[k] = (float)(48.0 * eps[k] * s6 * s6);
        h.c6[k] = (float)(24.0 * eps[k] * s6);
        h.e12[k] = (float)(4.0 * eps[k] * s6 * s6);
        h.e6[k] = (float)(4.0 * eps[k] * s6);
        h.sig2[k] = (float)s2;
        h.eps48[k] = (float)(48.0 * eps[k]);
        h.eps4[k] = (float)(4.0 * eps[k]);
        h.rc2[k] = (float)rc2;
        h.shift[k] = (float)sh;
        h.dsig2[k] = s2;
        h.deps48[k] = 48.0 * eps[k];
        h.deps4[k] = 4.0 * eps[k];
        h.drc2[k] = rc2;
        h.dshift[k] = sh;
        h.deps[k] = eps[k];
        h.dsig[k] = sigma[k];
    }
    CK(b, cudaMemcpyAsync(b->d_lj, &h, sizeof h, cudaMemcpyHostToDevice, b->stream));
    b->nt = nt;
    b->d.nt = nt;
    b->d.c1 = make_float4(h.c12[0], h.c6[0], h.e12[0], h.e6[0]);
    b->d.rc2_1 = h.rc2[0];
    b->d.esh_1 = h.shift[0];
    b->skin = skin;
    b->rl = rl;
    BoxDev& d = b->d;
    d.rl2 = rl * rl;
    d.rl2f = (float)(rl * rl);
    d.band = (float)(1.5e-4 * rl * rl);
    double thr = 0.5 * skin - 2e-6;
    d.disp_thr2 = thr > 0 ? (float)(thr * thr) : 0.0f;
    if (grid_changes) CKS(make_grid(b));
    b->lj_set = true;
    b->rec_valid = false;
    CKS(full_rebuild(b));
    CKS(leave(b));
    return MD_OK;
}

md_status md_set_thermostat(md_box* b, const double* T_bath, double rate, uint64_t seed)
{
    if (!b || !(rate >= 0.0) || !std::isfinite(rate) || (rate > 0.0 && !T_bath))
        return fail(b, MD_ERR_ARG, "md_set_thermostat: bad arguments");
    if (rate > 0.0)
        for (int r = 0; r < b->nrep; ++r)
            if (!(T_bath[r] > 0.0) || !std::isfinite(T_bath[r]))
                return fail(b, MD_ERR_ARG, "md_set_thermostat: T_bath must be positive");
    CKS(enter(b));
    if (rate > 0.0)
        CK(b, cudaMemcpyAsync(b->d_tstat_T, T_bath, sizeof(double) * b->nrep, cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaMemsetAsync(b->d_step_ctr, 0, sizeof(long long), b->stream));   // step index restarts at 0
    b->tstat_rate = rate;
    b->d.tstat_seed = seed;
    b->d.tstat_thr = 0u;   // set per dt by md_integrate
    b->rec_valid = false;
    invalidate_graphs(b);
    CKS(leave(b));   // T_bath may be pageable host memory
    return MD_OK;
}

md_status md_neighbour_update(md_box* b, int32_t force_rebuild, int32_t* rebuilt)
{
    if (!b || !b->lj_set) return fail(b, MD_ERR_ARG, "md_neighbour_update: md_set_lj not called");
    CKS(enter(b));
    std::vector<unsigned long long> before(b->nrep), after(b->nrep);
    CK(b, cudaMemcpyAsync(before.data(), b->d.nbuild, sizeof(unsigned long long) * b->nrep,
                          cudaMemcpyDeviceToHost, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));
    if (force_rebuild) CKS(full_rebuild(b));
    CK(b, cudaMemcpyAsync(after.data(), b->d.nbuild, sizeof(unsigned long long) * b->nrep,
                          cudaMemcpyDeviceToHost, b->stream));
    CKS(leave(b));
    if (rebuilt) {
        int k = 0;
        for (int r = 0; r < b->nrep; ++r) k += after[r] != before[r];
        *rebuilt = k;
    }
    return MD_OK;
}

md_status md_force(md_box* b, double* force_out, double* epot, double* virial)
{
    if (!b || !b->lj_set) return fail(b, MD_ERR_ARG, "md_force: md_set_lj not called");
    CKS(enter(b));
    CKS(ensure_thermo(b, 1));
    CKS(clear_err(b));
    CKS(enqueue_force(b, 1, b->d_thermo));
    if (force_out && b->ntot > 0) {
        size_t fb = sizeof(double) * 3 * (size_t)b->ntot;
        if (is_device_ptr(force_out)) {
            CK(b, launch_force_out(b->d, force_out, lch(b)));
        } else {
            CKS(ensure_stage(b, fb));
            CK(b, launch_force_out(b->d, static_cast<double*>(b->d_stage), lch(b)));
            CK(b, cudaMemcpyAsync(force_out, b->d_stage, fb, cudaMemcpyDeviceToHost, b->stream));
        }
    }
    std::vector<double> th(4 * (size_t)b->nrep);
    CK(b, cudaMemcpyAsync(th.data(), b->d_thermo, sizeof(double) * th.size(), cudaMemcpyDeviceToHost,
                          b->stream));
    int e2[3];
    CKS(read_err(b, e2));
    CKS(leave(b));
    for (int r = 0; r < b->nrep; ++r) {
        if (epot) epot[r] = th[4 * r + 0];
        if (virial) virial[r] = th[4 * r + 2];
    }
    if (e2[0] & LJ_ERRBIT_TIMEOUT) return fail(b, MD_ERR_TIMEOUT, "md_force: a device-side wait timed out");
    if (e2[0] & LJ_ERRBIT_NONFINITE) return fail(b, MD_ERR_NONFINITE, "md_force: non-finite force");
    return MD_OK;
}

md_status md_integrate(md_box* b, double dt, int64_t nsteps, int32_t ckpt_every, double* thermo_out)
{
    if (!b || !b->lj_set) return fail(b, MD_ERR_ARG, "md_integrate: md_set_lj not called");
    if (!(dt > 0.0) || nsteps < 0 || ckpt_every < 0) return fail(b, MD_ERR_ARG, "md_integrate: bad arguments");
    if (ckpt_every > 0 && nsteps % ckpt_every != 0)
        return fail(b, MD_ERR_ARG, "md_integrate: nsteps must be a multiple of ckpt_every");
    if (nsteps == 0) return MD_OK;
    if (ckpt_every > 0 && b->tstat_rate > 0.0)
        return fail(b, MD_ERR_ARG, "md_integrate: no recorded run with the thermostat on");
    CKS(enter(b));
    {
        // collision threshold of this dt: floor(rate dt 2^32), as a 32-bit word
        double t = std::floor(b->tstat_rate * dt * 4294967296.0);
        unsigned thr = !(t > 0.0) ? 0u : (t >= 4294967295.0 ? 4294967295u : (unsigned)t);
        if (thr != b->d.tstat_thr) {
            b->d.tstat_thr = thr;
            invalidate_graphs(b);
        }
    }
    const bool record = ckpt_every > 0;
    b->rec_valid = false;
    if (record) CKS(ckpt_setup(b, (int)(nsteps / ckpt_every)));
    const int energy = thermo_out ? 1 : 0;
    const int64_t chunk = record ? ckpt_every : b->chunk_steps;
    if (energy) CKS(ensure_thermo(b, std::min(nsteps, chunk)));
    bool out_dev = energy && is_device_ptr(thermo_out);
    int64_t done = 0;
    int retries = 0;
    while (done < nsteps) {
        int64_t n = std::min(chunk, nsteps - done);
        if (record) {
            // checkpoint boundary: fresh lists, then save the build state
            CKS(full_rebuild(b));
            CKS(ckpt_copy(b, (int)(done / ckpt_every), false));
        }
        b->fresh_abs = false;   // offsets advance; xabs keeps the last build
        CKS(clear_err(b));
        CKS(snapshot(b, false));
        cudaGraphExec_t g;
        CKS(get_graph(b, n, dt, energy, &g));
        CK(b, cudaGraphLaunch(g, b->stream));
        unsigned long long runs = 0;
        CK(b, cudaMemcpyAsync(&runs, b->d_cond_runs, sizeof runs, cudaMemcpyDeviceToHost, b->stream));
        int e2[3];
        CKS(read_err(b, e2));
        // rebuild sequences the step graph's IF nodes ran
        b->launches += (int64_t)(runs - b->cond_runs_seen) * rebuild_kernels(b);
        b->cond_runs_seen = runs;
        for (auto& ge : b->graphs)
            if (ge.exec == g) {
                b->launches += ge.kernels;
                for (size_t k = 0; k < ge.used.size(); ++k)
                    if (ge.used[k]) {
                        float ms = 0.f;
                        CK(b, cudaEventElapsedTime(&ms, ge.ev[2 * k], ge.ev[2 * k + 1]));
                        b->prof_ms[k % 4] += ms;
                        b->prof_n[k % 4] += 1;
                    }
            }
        if (e2[0] & (LJ_ERRBIT_CAPACITY | LJ_ERRBIT_TILE)) {
            if (++retries > 8) return fail(b, MD_ERR_CAPACITY, "md_integrate: list keeps overflowing");
            CKS(snapshot(b, true));
            if (e2[0] & LJ_ERRBIT_TILE) CKS(make_segments(b, true));
            if (e2[0] & LJ_ERRBIT_CAPACITY) {
                int K = round_up((int64_t)(e2[1] * 1.15) + 8, 8);
                CKS(alloc_lists(b, std::max(K, b->d.K + 8)));
            }
            CKS(full_rebuild(b));
            continue;
        }
        if (e2[0] & LJ_ERRBIT_TIMEOUT) {
            CKS(leave(b));
            return fail(b, MD_ERR_TIMEOUT, "md_integrate: a device-side wait timed out");
        }
        if (e2[0] & LJ_ERRBIT_NONFINITE) {
            CKS(leave(b));
            return fail(b, MD_ERR_NONFINITE, "md_integrate: non-finite force");
        }
        if (energy) {
            size_t cnt = (size_t)n * b->nrep * 4;
            double* dst = thermo_out + (size_t)done * b->nrep * 4;
            CK(b, cudaMemcpyAsync(dst, b->d_thermo, sizeof(double) * cnt,
                                  out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
        }
        done += n;
        b->steps += n;
    }
    if (record) {
        b->rec_valid = true;
        b->rec_serial += 1;
        b->rec_nsteps = nsteps;
        b->rec_k = ckpt_every;
        b->rec_C = (int)(nsteps / ckpt_every);
        b->rec_dt = dt;
    }
    CKS(leave(b));
    return MD_OK;
}

md_status md_adjoint(md_box* b, const double* lam_x_T, const double* lam_v_T, double* lam_x_0,
                     double* lam_v_0, double* dL_deps, double* dL_dsigma)
{
    if (!b) return MD_ERR_ARG;
    if (b->all_pairs) return fail(b, MD_ERR_ARG, "md_adjoint: not in the all-pairs form");
    if (!b->rec_valid || !b->lj_set) return fail(b, MD_ERR_STATE, "md_adjoint: no recorded forward run");
    if (!lam_x_T || !lam_v_T || !lam_x_0 || !lam_v_0) return fail(b, MD_ERR_ARG, "md_adjoint: null array");
    CKS(enter(b));
    const size_t n3 = 3 * (size_t)b->ntot, np = (size_t)b->np;
    const int k = b->rec_k, C = b->rec_C;
    const double h = b->rec_dt;
    const int P = b->nt * b->nt;
    if (!b->d_lx) {
        CKS(dev_alloc(b, &b->d_lx, n3));
        CKS(dev_alloc(b, &b->d_lv, n3));
        CKS(dev_alloc(b, &b->d_g, n3));
        CKS(dev_alloc(b, &b->d_u, np));
        CKS(dev_alloc(b, &b->d_theta, 2 * LJ_MAXT * LJ_MAXT));
        CKS(dev_alloc(b, &b->d_wts, 3));
        CKS(dev_alloc(b, &b->d_partg, 2 * (size_t)LJ_MAXT * LJ_MAXT * std::max<size_t>(1, b->chunks.size())));
    }
    size_t step_bytes = al256(np * 16) + 2 * al256(np * 4) + al256(np * (size_t)b->d.K * 4);
    if (b->tape_step_bytes != step_bytes || b->tape_cap < k + 1) {
        dev_release(b, b->d_tape);
        b->d_tape = nullptr;
        CKS(dev_alloc(b, &b->d_tape, step_bytes * (size_t)(k + 1), false));
        b->tape_step_bytes = step_bytes;
        b->tape_cap = k + 1;
    }
    const double wts[3] = {0.5 * h, h, 1.0};   // state weights, then the final reduction's
    CK(b, cudaMemcpyAsync(b->d_wts, wts, sizeof wts, cudaMemcpyHostToDevice, b->stream));
    CK(b, cudaMemsetAsync(b->d_theta, 0, sizeof(double) * 2 * LJ_MAXT * LJ_MAXT, b->stream));
    // parameter-gradient shares, accumulated over the whole reverse sweep
    CK(b, cudaMemsetAsync(b->d_partg, 0,
                          sizeof(double) * 2 * (size_t)LJ_MAXT * LJ_MAXT * std::max<size_t>(1, b->chunks.size()),
                          b->stream));
    const void *ix, *iv;
    CKS(ensure_stage(b, 2 * n3 * sizeof(double)));
    CKS(input_ptr(b, lam_x_T, n3 * sizeof(double), &ix, 0));
    CKS(input_ptr(b, lam_v_T, n3 * sizeof(double), &iv, n3 * sizeof(double)));
    CK(b, cudaMemcpyAsync(b->d_lx, ix, n3 * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    CK(b, cudaMemcpyAsync(b->d_lv, iv, n3 * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    CK(b, cudaStreamSynchronize(b->stream));   // host inputs staged before reuse
    // keep the current (end of run) state; restored at the end
    CKS(snapshot(b, false));
    Launch l = lch(b);
    Launch lf = lforce(b);
    // parameter-gradient rows: one per chunk, one per warp and chunk for one species
    const int nchunk = (int)b->chunks.size() * (P == 1 ? LJ_FORCE_WARPS : 1);
    const int twoP = 2 * P;
    // The replay of a segment (k recorded steps keeping the tape) and its
    // reverse sweep have the same launches for every segment: each is
    // captured once into a CUDA graph and launched per segment.  The reverse
    // sweep has four forms: the last segment also starts from the final
    // state's HVP, and the first weights its last term by h/2.
    struct Graphs {
        cudaGraphExec_t g[5] = {};
        int64_t kernels[5] = {};
        ~Graphs()
        {
            for (auto e : g)
                if (e) cudaGraphExecDestroy(e);
        }
    } graphs;
    auto capture = [&](int slot, auto&& fn) -> md_status {
        const int64_t l0 = b->launches;
        CK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        md_status st = fn();
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
        graphs.kernels[slot] = b->launches - l0;
        b->launches = l0;
        if (st != MD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess) return cuda_fail(b, ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&graphs.g[slot], graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(b, ce, "cudaGraphInstantiate");
        return MD_OK;
    };
    auto launch = [&](int slot) -> md_status {
        CK(b, cudaGraphLaunch(graphs.g[slot], b->stream));
        b->launches += graphs.kernels[slot];
        return MD_OK;
    };
    auto reverse = [&](bool last, bool first) -> md_status {
        for (int m = k; m >= 0; --m) {
            BoxDev v = tape_view(b, m);
            if (m == k) {
                if (!last) continue;   // this state's HVP was done at m = 0 of the next segment
                CK(b, launch_adj_pre(v, b->d_lx, b->d_lv, b->d_g, b->d_u, h, 0, l));
                CK(b, launch_hvp(v, b->d_u, b->d_lx, b->d_g, h, 0, b->d_wts, b->d_partg, lf));
            } else {
                CK(b, launch_adj_pre(v, b->d_lx, b->d_lv, b->d_g, b->d_u, h, 1, l));
                CK(b, launch_hvp(v, b->d_u, b->d_lx, b->d_g, h, 1, b->d_wts + ((first && m == 0) ? 0 : 1),
                                 b->d_partg, lf));
            }
            b->launches += 2;
        }
        return MD_OK;
    };
    for (int c = C - 1; c >= 0; --c) {
        // replay segment c, keeping every state's HVP inputs on the tape
        CKS(ckpt_copy(b, c, true));
        CKS(clear_err(b));
        CKS(replay_lists(b));
        CKS(tape_save(b, 0));
        if (!graphs.g[4]) CKS(capture(4, [&]() { return enqueue_steps(b, k, h, 0, nullptr, nullptr, true); }));
        CKS(launch(4));
        unsigned long long runs = 0;
        CK(b, cudaMemcpyAsync(&runs, b->d_cond_runs, sizeof runs, cudaMemcpyDeviceToHost, b->stream));
        int e2[3];
        CKS(read_err(b, e2));
        b->launches += (int64_t)(runs - b->cond_runs_seen) * rebuild_kernels(b);   // the replay's rebuilds
        b->cond_runs_seen = runs;
        if (e2[0]) return fail(b, MD_ERR_CAPACITY, "md_adjoint: replay of a segment failed");
        const int form = (c == C - 1 ? 1 : 0) | (c == 0 ? 2 : 0);
        if (!graphs.g[form]) CKS(capture(form, [&]() { return reverse(c == C - 1, c == 0); }));
        CKS(launch(form));
    }
    CK(b, launch_param_reduce(b->d_partg, nchunk, twoP, b->d_wts + 2, b->d_theta, b->stream));
    b->launches += 1;
    // outputs
    bool dx = is_device_ptr(lam_x_0), dv = is_device_ptr(lam_v_0);
    CK(b, cudaMemcpyAsync(lam_x_0, b->d_lx, n3 * sizeof(double), dx ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          b->stream));
    CK(b, cudaMemcpyAsync(lam_v_0, b->d_lv, n3 * sizeof(double), dv ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          b->stream));
    std::vector<double> th(2 * (size_t)P);
    CK(b, cudaMemcpyAsync(th.data(), b->d_theta, sizeof(double) * 2 * P, cudaMemcpyDeviceToHost, b->stream));
    // back to the end-of-run state
    CKS(snapshot(b, true));
    CKS(full_rebuild(b));
    b->fresh_abs = false;
    CKS(leave(b));
    const int nt = b->nt;
    std::vector<double> ge(P), gs(P);
    for (int a = 0; a < nt; ++a)
        for (int q = 0; q < nt; ++q) {
            int lo = std::min(a, q), hi = std::max(a, q);
            ge[a * nt + q] = th[lo * nt + hi];
            gs[a * nt + q] = th[P + lo * nt + hi];
        }
    if (dL_deps) {
        if (is_device_ptr(dL_deps)) CK(b, cudaMemcpy(dL_deps, ge.data(), sizeof(double) * P, cudaMemcpyHostToDevice));
        else std::memcpy(dL_deps, ge.data(), sizeof(double) * P);
    }
    if (dL_dsigma) {
        if (is_device_ptr(dL_dsigma)) CK(b, cudaMemcpy(dL_dsigma, gs.data(), sizeof(double) * P, cudaMemcpyHostToDevice));
        else std::memcpy(dL_dsigma, gs.data(), sizeof(double) * P);
    }
    return MD_OK;
}

md_status md_pair_hist(md_box* b, int32_t nbins, double rhist, double width, double rmax, const double* coef,
                       double* hist, double* grad)
{
    if (!b || !b->lj_set || nbins < 1 || nbins > 256 || !(rhist > 0) || !(width > 0) || !(rmax > 0))
        return fail(b, MD_ERR_ARG, "md_pair_hist: bad arguments");
    if (rmax > b->rl) return fail(b, MD_ERR_ARG, "md_pair_hist: rmax beyond the list radius");
    if (b->all_pairs) return fail(b, MD_ERR_ARG, "md_pair_hist: not in the all-pairs form (no lists)");
    CKS(enter(b));
    // the lists must hold every pair below rmax at the current positions
    if (!b->fresh_abs) CKS(full_rebuild(b));
    const size_t nh = (size_t)b->nrep * nbins;
    if (b->hist_cap < nbins) {
        dev_release(b, b->d_parth);
        dev_release(b, b->d_hist);
        CKS(dev_alloc(b, &b->d_parth, (size_t)nbins * std::max<size_t>(1, b->chunks.size())));
        CKS(dev_alloc(b, &b->d_hist, (size_t)b->nrep * nbins));
        b->hist_cap = nbins;
    }
    if (hist) {
        CK(b, launch_pair_hist(b->d, nbins, rhist, width, rmax, b->d_parth, b->d_hist, lch(b)));
        CK(b, cudaMemcpyAsync(hist, b->d_hist, sizeof(double) * nh,
                              is_device_ptr(hist) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
        b->launches += 2;
    }
    if (grad && coef && b->ntot > 0) {
        const size_t gb = sizeof(double) * 3 * (size_t)b->ntot;
        CKS(ensure_stage(b, gb + sizeof(double) * nh + 256));
        const void* dc;
        CKS(input_ptr(b, coef, sizeof(double) * nh, &dc, al256(gb)));
        double* dg = is_device_ptr(grad) ? grad : reinterpret_cast<double*>(b->d_stage);
        CK(b, launch_pair_hist_grad(b->d, nbins, rhist, width, rmax, static_cast<const double*>(dc), dg, lch(b)));
        b->launches += 1;
        if (dg != grad) CK(b, cudaMemcpyAsync(grad, dg, gb, cudaMemcpyDeviceToHost, b->stream));
    }
    CKS(leave(b));
    return MD_OK;
}

md_status md_get_state(md_box* b, double* pos, double* vel, int32_t* image)
{
    if (!b) return MD_ERR_ARG;
    if (b->ntot == 0) return MD_OK;
    if (!b->binned) return fail(b, MD_ERR_ARG, "md_get_state: md_set_lj not called");
    CKS(enter(b));
    size_t pb = sizeof(double) * 3 * (size_t)b->ntot, ib = sizeof(int) * 3 * (size_t)b->ntot;
    bool dp = is_device_ptr(pos), dv = is_device_ptr(vel), di = is_device_ptr(image);
    CKS(ensure_stage(b, 2 * pb + ib));
    char* st = static_cast<char*>(b->d_stage);
    double* tp = pos ? (dp ? pos : reinterpret_cast<double*>(st)) : nullptr;
    double* tv = vel ? (dv ? vel : reinterpret_cast<double*>(st + pb)) : nullptr;
    int* ti = image ? (di ? image : reinterpret_cast<int*>(st + 2 * pb)) : nullptr;
    CK(b, launch_download(b->d, tp, tv, ti, lch(b)));
    if (pos && !dp) CK(b, cudaMemcpyAsync(pos, tp, pb, cudaMemcpyDeviceToHost, b->stream));
    if (vel && !dv) CK(b, cudaMemcpyAsync(vel, tv, pb, cudaMemcpyDeviceToHost, b->stream));
    if (image && !di) CK(b, cudaMemcpyAsync(image, ti, ib, cudaMemcpyDeviceToHost, b->stream));
    CKS(leave(b));
    return MD_OK;
}

md_status md_set_state(md_box* b, const double* pos, const double* vel)
{
    if (!b || (!pos && b->ntot > 0)) return MD_ERR_ARG;
    if (b->ntot == 0) return MD_OK;
    CKS(enter(b));
    size_t pb = sizeof(double) * 3 * (size_t)b->ntot;
    CKS(ensure_stage(b, 3 * pb));
    char* st = static_cast<char*>(b->d_stage);
    const void* dpos;
    CKS(input_ptr(b, pos, pb, &dpos, 0));
    const double* dvel = nullptr;
    if (vel) {
        const void* v;
        CKS(input_ptr(b, vel, pb, &v, pb));
        dvel = static_cast<const double*>(v);
    } else if (b->binned) {
        // keep the velocities: bring them to user order first
        double* tv = reinterpret_cast<double*>(st + 2 * pb);
        CK(b, launch_download(b->d, nullptr, tv, nullptr, lch(b)));
        dvel = tv;
    }
    if (dpos == st + 2 * pb) return fail(b, MD_ERR_ARG, "internal staging overlap");
    CK(b, launch_upload(b->d, static_cast<const double*>(dpos), dvel, b->d_type_user,
                        (vel || b->binned) ? 1 : 0, lch(b)));
    b->fresh_abs = true;
    b->rec_valid = false;
    if (b->lj_set) CKS(full_rebuild(b));
    CKS(leave(b));
    return MD_OK;
}

md_status md_get_nlist(md_box* b, int32_t* count, int64_t* nbr, int64_t cap, double* pos)
{
    if (!b || !count || (nbr && cap < 1)) return MD_ERR_ARG;
    if (!b->lj_set) return fail(b, MD_ERR_ARG, "md_get_nlist: md_set_lj not called");
    if (b->all_pairs) return fail(b, MD_ERR_ARG, "md_get_nlist: the all-pairs form has no lists");
    if (b->ntot == 0) return MD_OK;
    CKS(enter(b));
    size_t cb = sizeof(int) * (size_t)b->ntot;
    size_t nb = nbr ? sizeof(int64_t) * (size_t)b->ntot * (size_t)cap : 0;
    size_t pb = pos ? sizeof(double) * 3 * (size_t)b->ntot : 0;
    CKS(ensure_stage(b, cb + nb + pb + 512));
    char* st = static_cast<char*>(b->d_stage);
    int* tc = reinterpret_cast<int*>(st);
    long long* tn = nbr ? reinterpret_cast<long long*>(st + ((cb + 255) & ~(size_t)255)) : nullptr;
    double* tp = pos ? reinterpret_cast<double*>(st + ((cb + 255) & ~(size_t)255) + ((nb + 255) & ~(size_t)255))
                     : nullptr;
    CK(b, launch_get_nlist(b->d, tc, tn, (long long)cap, tp, lch(b)));
    std::vector<int> hc(b->ntot);
    CK(b, cudaMemcpyAsync(hc.data(), tc, cb, cudaMemcpyDeviceToHost, b->stream));
    if (nbr) CK(b, cudaMemcpyAsync(nbr, tn, nb, is_device_ptr(nbr) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (pos) CK(b, cudaMemcpyAsync(pos, tp, pb, is_device_ptr(pos) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    CKS(leave(b));
    int mx = 0;
    for (int v : hc) mx = std::max(mx, v);
    if (is_device_ptr(count)) {
        CK(b, cudaMemcpy(count, hc.data(), cb, cudaMemcpyHostToDevice));
    } else {
        std::memcpy(count, hc.data(), cb);
    }
    if (mx > b->d.K) return fail(b, MD_ERR_CAPACITY, "md_get_nlist: list truncated at capacity");
    if (nbr && mx > cap) return fail(b, MD_ERR_CAPACITY, "md_get_nlist: cap too small");
    return MD_OK;
}

md_status md_get_info(md_box* b, md_info* out)
{
    if (!b || !out) return MD_ERR_ARG;
    md_info i{};
    i.n_total = b->ntot;
    i.nrep = b->nrep;
    i.ntypes = b->nt;
    i.capacity = b->d.K;
    i.precision = b->prec;
    i.ncell_total = b->d.ncell;
    i.steps = b->steps;
    int64_t bytes = 0;
    for (auto& a : b->allocs) bytes += (int64_t)a.bytes;
    i.device_bytes = bytes;
    i.rlist = b->rl;
    i.launches = b->launches;
    i.record_id = b->rec_valid ? b->rec_serial : 0;
    if (b->lj_set) {
        std::vector<unsigned long long> nb(b->nrep);
        CK(b, cudaSetDevice(b->device));
        CK(b, cudaMemcpyAsync(nb.data(), b->d.nbuild, sizeof(unsigned long long) * b->nrep,
                              cudaMemcpyDeviceToHost, b->stream));
        CK(b, cudaStreamSynchronize(b->stream));
        for (auto v : nb) i.rebuilds += (int64_t)v;
        std::vector<int> cnt(b->np);
        CK(b, cudaMemcpyAsync(cnt.data(), b->d.nbr_count, sizeof(int) * b->np, cudaMemcpyDeviceToHost,
                              b->stream));
        CK(b, cudaStreamSynchronize(b->stream));
        for (int c : cnt) i.list_entries += c;
    }
    *out = i;
    return MD_OK;
}

md_status md_set_profiling(md_box* b, int32_t on)
{
    if (!b) return MD_ERR_ARG;
    b->profiling = on != 0;
    for (int k = 0; k < 4; ++k) {
        b->prof_ms[k] = 0.0;
        b->prof_n[k] = 0;
    }
    invalidate_graphs(b);
    return MD_OK;
}

md_status md_get_profile(md_box* b, double* ms, int64_t* launches)
{
    if (!b) return MD_ERR_ARG;
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = b->prof_ms[k];
        if (launches) launches[k] = b->prof_n[k];
    }
    return MD_OK;
}

md_status md_get_tuning(md_box* b, int32_t t[4])
{
    if (!b || !t) return MD_ERR_ARG;
    t[0] = b->force_per_sm;
    t[1] = b->list_per_sm;
    t[2] = b->seg_cells;
    t[3] = b->min_capacity;
    return MD_OK;
}

md_status md_set_tuning(md_box* b, const int32_t t[4])
{
    if (!b || !t || t[0] < 0 || t[0] > 32 || t[1] < 0 || t[1] > 32 || t[2] < 0 || t[2] > LJ_SEG_MAX_CELLS ||
        t[3] < 0)
        return fail(b, MD_ERR_ARG, "md_set_tuning: values out of range");
    const bool seg_changed = t[2] != b->seg_cells;
    b->force_per_sm = t[0];
    b->list_per_sm = t[1];
    b->seg_cells = t[2];
    b->min_capacity = t[3];
    invalidate_graphs(b);
    if (!b->lj_set) return MD_OK;
    if (t[3] > 0 || seg_changed) {
        CKS(enter(b));
        if (seg_changed) CKS(make_segments(b, false));
        if (t[3] > 0) CKS(alloc_lists(b, round_up(t[3], 8)));   // 16-byte list rows
        CKS(full_rebuild(b));
        CKS(leave(b));
    }
    return MD_OK;
}

md_status md_autotune(md_box* b, int32_t reps, int32_t t[4])
{
    if (!b || !b->lj_set || reps < 1) return fail(b, MD_ERR_ARG, "md_autotune: md_set_lj not called");
    if (b->all_pairs) return fail(b, MD_ERR_ARG, "md_autotune: not in the all-pairs form");
    CKS(enter(b));
    // pair-force grid of the chunk kernel: blocks per SM (the tiled kernel
    // runs its resident blocks)
    const int fcand[] = {2, 3, 4, 6, 8, 12, 16, 24, 32};
    int best_f = b->force_per_sm > 0 ? b->force_per_sm : 6;
    float best_ft = 1e30f;
    for (int c : fcand) {
        if (b->d.force_tiles) break;
        b->force_per_sm = c;
        float ms = 0.f;
        CKS(time_launches(b, reps, [&]() -> md_status { return enqueue_force(b, 1, nullptr); }, &ms));
        if (ms < best_ft) {
            best_ft = ms;
            best_f = c;
        }
    }
    b->force_per_sm = best_f;
    // list build: segment length x blocks per SM, timed as forced rebuilds
    int s0 = b->reps.empty() ? 4 : b->reps[0].S;
    int best_s = s0, best_l = 6;
    float best_lt = 1e30f;
    const int lcand[] = {3, 4, 6, 8, 12};
    for (int S = std::max(1, s0 - 2); S <= std::min(LJ_SEG_MAX_CELLS, s0 + 2); ++S) {
        b->seg_cells = S;
        CKS(make_segments(b, false));
        for (int lc : lcand) {
            b->list_per_sm = lc;
            float ms = 0.f;
            md_status st = time_launches(b, reps, [&]() -> md_status {
                CKS(set_all_rebuild(b));
                return enqueue_rebuild(b, b->fresh_abs ? 1 : 0);
            }, &ms);
            if (st != MD_OK) return st;
            int e2[3];
            CKS(read_err(b, e2));
            if (e2[0] & (LJ_ERRBIT_TILE | LJ_ERRBIT_CAPACITY)) {
                CKS(clear_err(b));
                continue;   // this segment length overflows a tile: not a candidate
            }
            if (ms < best_lt) {
                best_lt = ms;
                best_s = S;
                best_l = lc;
            }
        }
    }
    b->seg_cells = best_s;
    b->list_per_sm = best_l;
    CKS(make_segments(b, false));
    CKS(full_rebuild(b));
    // cell layout: a step's cost (one force evaluation, plus one list build
    // spread over the observed steps per build) for each candidate
    {
        unsigned long long nb = 0;
        std::vector<unsigned long long> nbv(b->nrep);
        CK(b, cudaMemcpyAsync(nbv.data(), b->d.nbuild, sizeof(unsigned long long) * b->nrep, cudaMemcpyDeviceToHost,
                              b->stream));
        CK(b, cudaStreamSynchronize(b->stream));
        for (auto v : nbv) nb = std::max(nb, v);
        const double spb = (b->steps > 0 && nb > 2) ? std::max(1.0, (double)b->steps / (double)(nb - 2)) : 10.0;
        const double scales[4] = {1.0, 1.08, 1.15, 1.22};
        double best_cost = 1e300, best_scale = b->cell_scale;
        int best_order = b->order;
        // the list-build kernel too, unless the caller fixed it
        const int fixed_kind = b->list_kernel;
        const int kinds[2] = {MD_LIST_LANES, MD_LIST_QUADS};
        const int nkind = fixed_kind == MD_LIST_AUTO ? 2 : 1;
        int best_kind = fixed_kind;
        for (int ki = 0; ki < nkind; ++ki)
        for (double sc : scales)
            for (int od = 0; od < 2; ++od) {
                if (fixed_kind == MD_LIST_AUTO && b->list_kernel != kinds[ki]) {
                    b->list_kernel = kinds[ki];
                    invalidate_graphs(b);
                }
                const md_status st = set_layout(b, sc, od);
                if (st == MD_ERR_CAPACITY) continue;   // its tiles overflow: not a candidate
                if (st != MD_OK) return st;
                float ms_f = 0.f, ms_b = 0.f;
                CKS(time_launches(b, reps, [&]() -> md_status { return enqueue_force(b, 1, nullptr); }, &ms_f));
                CKS(time_launches(b, reps, [&]() -> md_status {
                    CKS(set_all_rebuild(b));
                    return enqueue_rebuild(b, b->fresh_abs ? 1 : 0);
                }, &ms_b));
                int e2[3];
                CKS(read_err(b, e2));
                if (e2[0] & (LJ_ERRBIT_TILE | LJ_ERRBIT_CAPACITY)) {
                    CKS(clear_err(b));
                    CKS(full_rebuild(b));   // regrow, then time this layout again
                    CKS(time_launches(b, reps, [&]() -> md_status {
                        CKS(set_all_rebuild(b));
                        return enqueue_rebuild(b, b->fresh_abs ? 1 : 0);
                    }, &ms_b));
                }
                const double cost = ms_f + ms_b / spb;
                if (cost < best_cost) {
                    best_cost = cost;
                    best_scale = sc;
                    best_order = od;
                    best_kind = b->list_kernel;
                }
            }
        if (b->list_kernel != best_kind) {
            b->list_kernel = best_kind;
            invalidate_graphs(b);
            // a layout the other kernel refuses is re-gridded by set_layout below
            if (b->cell_scale == best_scale && b->order == best_order) CKS(full_rebuild(b));
        }
        CKS(set_layout(b, best_scale, best_order));
        // the list build's grid again, at the chosen layout and kernel
        float best_g = 1e30f;
        int best_gl = b->list_per_sm;
        for (int lc : {3, 4, 6, 8, 12, 16, 24}) {
            b->list_per_sm = lc;
            float ms = 0.f;
            CKS(time_launches(b, reps, [&]() -> md_status {
                CKS(set_all_rebuild(b));
                return enqueue_rebuild(b, b->fresh_abs ? 1 : 0);
            }, &ms));
            int e2[3];
            CKS(read_err(b, e2));
            if (e2[0] & (LJ_ERRBIT_TILE | LJ_ERRBIT_CAPACITY)) {
                CKS(clear_err(b));
                continue;
            }
            if (ms < best_g) {
                best_g = ms;
                best_gl = lc;
            }
        }
        b->list_per_sm = best_gl;
        invalidate_graphs(b);
        CKS(full_rebuild(b));
    }
    // the FP32 list-form force kernel, unless the caller fixed it: both timed
    // at the chosen layout, the faster kept (md_get_force_kernel reads it)
    if (b->force_kernel == MD_FORCE_AUTO && !b->all_pairs && b->prec != MD_PREC_FP64) {
        const int kinds[2] = {MD_FORCE_CHUNKS, MD_FORCE_TILES};
        float tk[2] = {1e30f, 1e30f};
        for (int i = 0; i < 2; ++i) {
            b->force_kernel = kinds[i];
            apply_force_kernel(b);
            CKS(time_launches(b, reps, [&]() -> md_status { return enqueue_force(b, 1, nullptr); }, &tk[i]));
        }
        b->force_kernel = tk[1] < tk[0] ? MD_FORCE_TILES : MD_FORCE_CHUNKS;
        apply_force_kernel(b);
        invalidate_graphs(b);
        CKS(enqueue_force(b, 1, nullptr));   // the box's forces from the kept kernel
    }
    CKS(leave(b));
    return md_get_tuning(b, t);
}

md_status md_set_layout(md_box* b, double cell_scale, int32_t order)
{
    if (!b || !(cell_scale >= 1.0) || !std::isfinite(cell_scale) || order < 0 || order > 1)
        return fail(b, MD_ERR_ARG, "md_set_layout: cell_scale must be >= 1 and order 0 or 1");
    if (b->all_pairs) return fail(b, MD_ERR_ARG, "md_set_layout: not in the all-pairs form");
    if (!b->lj_set) {   // applied by md_set_lj
        b->cell_scale = cell_scale;
        b->order = order;
        b->d.order = order;
        return MD_OK;
    }
    CKS(enter(b));
    CKS(set_layout(b, cell_scale, order));
    CKS(leave(b));
    return MD_OK;
}

md_status md_set_list_kernel(md_box* b, int32_t kind)
{
    if (!b || kind < MD_LIST_AUTO || kind > MD_LIST_LANES)
        return fail(b, MD_ERR_ARG, "md_set_list_kernel: kind must be 0, 1 or 2");
    if (kind != b->list_kernel) {
        b->list_kernel = kind;
        invalidate_graphs(b);
    }
    return MD_OK;
}

md_status md_set_force_kernel(md_box* b, int32_t kind)
{
    if (!b || kind < MD_FORCE_AUTO || kind > MD_FORCE_TILES)
        return fail(b, MD_ERR_ARG, "md_set_force_kernel: kind must be 0, 1 or 2");
    if (kind != b->force_kernel) {
        b->force_kernel = kind;
        apply_force_kernel(b);
        invalidate_graphs(b);
    }
    return MD_OK;
}

md_status md_get_force_kernel(md_box* b, int32_t* kind)
{
    if (!b || !kind) return MD_ERR_ARG;
    *kind = b->force_kernel;
    return MD_OK;
}

md_status md_set_graph_conditional(md_box* b, int32_t on)
{
    if (!b || on < 0 || on > 1) return fail(b, MD_ERR_ARG, "md_set_graph_conditional: on must be 0 or 1");
    if ((on != 0) != b->use_cond) {
        b->use_cond = on != 0;
        invalidate_graphs(b);
    }
    return MD_OK;
}

md_status md_get_graph_conditional(md_box* b, int32_t* on)
{
    if (!b || !on) return MD_ERR_ARG;
    *on = b->use_cond ? 1 : 0;
    return MD_OK;
}

md_status md_get_list_kernel(md_box* b, int32_t* kind)
{
    if (!b || !kind) return MD_ERR_ARG;
    *kind = b->list_kernel;
    return MD_OK;
}

md_status md_get_layout(md_box* b, double* cell_scale, int32_t* order)
{
    if (!b) return MD_ERR_ARG;
    if (cell_scale) *cell_scale = b->cell_scale;
    if (order) *order = b->order;
    return MD_OK;
}

}  // extern "C"

// ==========================================================================
// Force and energy evaluation that allocates nothing.
//
// For callers that must not allocate device memory at the point of the call:
// code running while a memory pool is frozen or capped, a host that shares
// the GPU with a framework owning all of its memory, or a real-time loop that
// may not block on an allocator.  The per-chunk energy/virial partial sums
// and the per-replica totals (the only scratch of this computation beyond
// what the box already owns) live in the file-scope array below instead of
// box-owned buffers that md_force may grow lazily.
// ==========================================================================
#include <mutex>

#define LJMD_NOALLOC_DOUBLES (1 << 19)   // 4 MiB of FP64 scratch, per device

// One copy per device that loads this library, held until process exit.
static __device__ __align__(256) double g_noalloc_scratch[LJMD_NOALLOC_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 128;
double* g_noalloc_dev[kMaxDevices] = {};   // device address of the array, per device
}  // namespace

extern "C" md_status md_force_noalloc(md_box* b, double* force_out, double* epot, double* virial)
{
    if (!b) return MD_ERR_ARG;
    // the chunk kernels always (their shares are per warp, not per particle)
    BoxDev v = b->d;
    v.force_tiles = 0;   // same share layout per chunk as the FP32 list kernels
    const size_t nchunk = b->chunks.size();
    const size_t nshare = 2 * (size_t)v.pf_stride * nchunk;   // (E_pot, W) shares
    const size_t need = nshare + 4 * (size_t)b->nrep;
    if (need > (size_t)LJMD_NOALLOC_DOUBLES) {
        char msg[240];
        snprintf(msg, sizeof msg,
                 "md_force_noalloc: box needs %zu scratch doubles (16 per 128 particles with FP32 forces, 8 "
                 "all-FP64, 2 for all pairs, + 4 per replica); the static scratch holds %d",
                 need, LJMD_NOALLOC_DOUBLES);
        return fail(b, MD_ERR_ARG, msg);
    }
    if (!b->lj_set) return fail(b, MD_ERR_ARG, "md_force_noalloc: md_set_lj not called");
    if (force_out && !is_device_ptr(force_out))
        return fail(b, MD_ERR_ARG, "md_force_noalloc: force_out must be device memory of the box's GPU");
    if (b->device < 0 || b->device >= kMaxDevices) return fail(b, MD_ERR_ARG, "md_force_noalloc: device ordinal");
    double* scratch = nullptr;
    {
        // first call on this device: look up the array's device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_dev[b->device]) {
            CK(b, cudaSetDevice(b->device));
            void* p = nullptr;
            CK(b, cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_dev[b->device] = static_cast<double*>(p);
        }
        scratch = g_noalloc_dev[b->device];
    }
    CKS(enter(b));
    v.part_f = scratch;                       // every chunk's shares are overwritten
    double* th = scratch + nshare;            // nrep x (E_pot, E_kin, W, T), overwritten
    CKS(clear_err(b));
    Launch lf = lforce(b);
    if (b->d.force_tiles) {   // the chunk kernel's grid
        const int per_sm = b->force_per_sm > 0 ? b->force_per_sm : 6;
        lf.grid = std::max(1, std::min((int)v.nchunk, b->nsm * per_sm));
    }
    CK(b, launch_force(v, 1, lf));
    CK(b, launch_thermo(v, th, 0, lthermo(b)));
    if (force_out && b->ntot > 0) CK(b, launch_force_out(b->d, force_out, lch(b)));
    if (epot)
        CK(b, cudaMemcpy2DAsync(epot, sizeof(double), th + 0, 4 * sizeof(double), sizeof(double), b->nrep,
                                is_device_ptr(epot) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    if (virial)
        CK(b, cudaMemcpy2DAsync(virial, sizeof(double), th + 2, 4 * sizeof(double), sizeof(double), b->nrep,
                                is_device_ptr(virial) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                b->stream));
    int e2[3];
    CKS(read_err(b, e2));
    CKS(leave(b));
    if (e2[0] & LJ_ERRBIT_NONFINITE) return fail(b, MD_ERR_NONFINITE, "md_force_noalloc: non-finite force");
    return MD_OK;
}
