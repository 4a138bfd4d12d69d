// k_rebuild.cu -- particle binning, counting sort by cell and Verlet-list build.
//
// Sec. 3 (Code structure): Verlet neighbour lists are built efficiently from
// a spatial decomposition of the particles ("particle binning"); Sec. 5
// (Truncated Force Performance Study): the list update is ~30 % of the run
// time.  A rebuild of replica r runs only when rep_needs_rebuild(r) (the skin
// rule: some particle moved more than skin/2 since the last build, or the
// host forced it); every kernel here tests that flag per work item, so the
// whole sequence can sit in a CUDA graph and cost one early exit per kernel
// when no replica needs it.
//
// Sequence: k_bin (new cell of every particle, counts) -> k_scan_tiles +
// k_scan_add (exclusive scan of the counts per replica) -> k_scatter (slot
// per particle) -> k_sortgather (order inside each cell by FP32 z offset,
// ties by user index, so the layout is a deterministic function of the
// positions; gather into the sorted arrays) -> k_nlist (27-cell search,
// each neighbour cell narrowed to its candidates within reach along z).
#include <climits>

#include "ljmd_internal.cuh"

namespace {

constexpr int kScanTile = 4096;   // cells per scan tile

__device__ __forceinline__ int cell_coords(const RepDev& R, int gc, int& cx, int& cy)
{
    int local = gc - R.cell_off;
    cx = local % R.nc[0];
    int t = local / R.nc[0];
    cy = t % R.nc[1];
    return t / R.nc[1];
}

// Cell (chunk) t of the concatenation of the rebuilding replicas' cells
// (particle chunks), from k_list_work's lists; kr is the replica index of the
// caller's previous t (t only grows).
__device__ __forceinline__ int work_cell(const BoxDev& b, int t, int& kr)
{
    while (t >= b.lw_off[kr + 1]) ++kr;
    return b.rep[b.lw_rep[kr]].cell_off + (t - b.lw_off[kr]);
}
__device__ __forceinline__ int work_chunk(const BoxDev& b, int t, int& kr)
{
    while (t >= b.lw_coff[kr + 1]) ++kr;
    return b.rep[b.lw_rep[kr]].chunk_off + (t - b.lw_coff[kr]);
}

// 8-byte component c of particle p of an integrator array in the layout of
// the box precision (FP64: one double; DS: hi/lo floats in two planes).
__device__ __forceinline__ void copy_acc(const BoxDev& b, double* dst, const double* src, int c,
                                         int q, int p)
{
    if (b.prec == 0) {
        const float* s = reinterpret_cast<const float*>(src);
        float* d = reinterpret_cast<float*>(dst);
        d[c * b.np + q] = s[c * b.np + p];
        d[3 * b.np + c * b.np + q] = s[3 * b.np + c * b.np + p];
    } else {
        dst[c * b.np + q] = src[c * b.np + p];
    }
}

// ---------------------------------------------------------------------------
// k_bin: new cell of every particle of a rebuilding replica, its offset from
// the new cell's centre (offB, the state's layout), its wrapped FP64 position
// (xabsB, the positions the lists are decided for) and the old-order copies
// used by the gather.
//
// Steady state (double-single state, positions held as cell + offset): the
// move to a neighbour cell is read off the FP32 offset (|o| >= half an edge)
// and the new offset is o - d * edge in double-single arithmetic, so the
// only FP64 work is forming the position x = centre + o.  A particle that
// crosses the box, moves more than one cell, or sits in a boundary cell with
// x outside [0, L) at FP64 rounding, takes the FP64 path of a build from
// positions: wrap x into [0, L), cell = floor(x / edge), offset = x - centre.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_from_x(const BoxDev& b, const RepDev& R, double* x, int* im, int* q)
{
    for (int c = 0; c < 3; ++c) {
        const double L = R.L[c];
        // floor(x / L); the FP64 division (slow on this GPU) only where
        // the quotient can round to 1 or more, or x is negative
        const double f = (x[c] >= 0.0 && x[c] < R.wrap_hi[c]) ? 0.0 : floor(x[c] / L);
        if (f != 0.0) {
            x[c] = x[c] - L * f;
            im[c] += (int)f;
        }
        const int qc = (int)(x[c] * R.inv_ell[c]);
        q[c] = qc < 0 ? 0 : (qc >= R.nc[c] ? R.nc[c] - 1 : qc);
    }
}

// offset of x from the centre of cell q, in the state's layout (the centre
// rounded on its own, no FMA with the subtraction)
__device__ __forceinline__ void store_offB(const BoxDev& b, const RepDev& R, int p, const double* x, const int* q)
{
    for (int c = 0; c < 3; ++c) {
        const double o = x[c] - __dmul_rn((double)q[c] + 0.5, R.ell[c]);
        if (b.prec == 0) {
            float h, l;
            ds_from_double(o, h, l);
            float* ob = reinterpret_cast<float*>(b.offB);
            ob[c * b.np + p] = h;
            ob[3 * b.np + c * b.np + p] = l;
        } else {
            b.offB[c * b.np + p] = o;
        }
    }
}

__global__ void __launch_bounds__(LJ_CHUNK) k_bin(BoxDev b, int from_abs)
{
    if (!box_needs_rebuild(b)) return;
    const int tot = b.lw_coff[b.lw_hdr[0]];
    int kr = 0;
    for (int t = blockIdx.x; t < tot; t += gridDim.x) {
        const int w = work_chunk(b, t, kr);
        int4 ch = b.chunk[w];
        int r = ch.x;
        int p = ch.y + (int)threadIdx.x;
        const bool act = p < ch.z;   // every lane reaches the warp-wide count below
        if (!act) p = ch.y;
        const RepDev& R = b.rep[r];
        double x[3];
        int im[3], q[3];
        for (int c = 0; c < 3; ++c) im[c] = b.img[c * b.np + p];
        if (from_abs) {
            for (int c = 0; c < 3; ++c) x[c] = b.xabs[c * b.np + p];
            bin_from_x(b, R, x, im, q);
            if (act) store_offB(b, R, p, x, q);
        } else {
            int cx, cy;
            const int cz = cell_coords(R, b.cell[p], cx, cy);
            const int cc[3] = {cx, cy, cz};
            bool slow = b.prec != 0;
            float nh[3], nl[3];
            for (int c = 0; c < 3; ++c) {
                double o;
                if (b.prec == 0) {
                    const float* s = reinterpret_cast<const float*>(b.off);
                    const float h = s[c * b.np + p], l = s[3 * b.np + c * b.np + p];
                    o = (double)h + (double)l;
                    // the neighbour cell the FP32 offset lies in (at most one away)
                    const float hh = 0.5f * R.ellf[c];
                    const int d = h >= hh ? 1 : (h < -hh ? -1 : 0);
                    const int qc = cc[c] + d;
                    slow = slow || fabsf(h) >= 3.f * hh || qc < 0 || qc >= R.nc[c];
                    q[c] = qc;
                    // o - d * edge, double-single (d * ellf is exact)
                    float sh = h, sl = l;
                    ds_add_ds(sh, sl, -(float)d * R.ellf[c], -(float)d * R.ell_lo[c]);
                    nh[c] = sh;
                    nl[c] = sl;
                } else {
                    o = b.off[c * b.np + p];
                }
                x[c] = __dmul_rn((double)cc[c] + 0.5, R.ell[c]) + o;
                // a boundary cell: the position must still be inside [0, L)
                if ((cc[c] == 0 || cc[c] == R.nc[c] - 1) && !(x[c] >= 0.0 && x[c] < R.wrap_hi[c])) slow = true;
            }
            if (slow) {
                bin_from_x(b, R, x, im, q);
                if (act) store_offB(b, R, p, x, q);
            } else if (act) {
                float* ob = reinterpret_cast<float*>(b.offB);
                for (int c = 0; c < 3; ++c) {
                    ob[c * b.np + p] = nh[c];
                    ob[3 * b.np + c * b.np + p] = nl[c];
                }
            }
        }
        int gc = R.cell_off + q[0] + R.nc[0] * (q[1] + R.nc[1] * q[2]);
        if (act)
            for (int c = 0; c < 3; ++c) {
                b.xabsB[c * b.np + p] = x[c];
                b.imgB[c * b.np + p] = im[c];
                copy_acc(b, b.velB, b.vel, c, p, p);
            }
        if (act) {
            b.uidB[p] = b.uid[p];
            b.typeB[p] = b.type[p];
            b.cellB[p] = gc;
        }
        // warp-aggregated count: particles arrive in cell order, so a warp's
        // lanes share one or two cells; one atomic per distinct cell
        const int key = act ? gc : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (act && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&b.cell_count[gc], __popc(peers));
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of cell counts inside each replica, in two passes over
// tiles of kScanTile cells: k_scan_tiles writes the tile-local prefix into
// cell_start and the tile total into tile_sum; k_scan_add adds the totals of
// the replica's earlier tiles plus the replica's first slot.
// tiles[t] = (rep, first cell, end cell, first tile of the replica).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_excl_scan(int v, int* s_warp, int& total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int x = lane < nw ? s_warp[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) s_warp[lane] = xi - x;   // exclusive warp offsets
        if (lane == nw - 1) s_warp[32] = xi;    // block total
    }
    __syncthreads();
    int r = incl - v + s_warp[warp];
    total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(BoxDev b, const int4* tiles, int ntiles,
                                                      int* tile_sum)
{
    if (!box_needs_rebuild(b)) return;
    __shared__ int s_warp[33];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int4 tl = tiles[t];
        if (!rep_needs_rebuild(b, tl.x)) continue;   // block-uniform
        int carry = 0;
        for (int base = tl.y; base < tl.z; base += blockDim.x) {
            int c = base + (int)threadIdx.x;
            int v = c < tl.z ? b.cell_count[c] : 0;
            int total;
            int ex = block_excl_scan(v, s_warp, total);
            if (c < tl.z) b.cell_start[c] = carry + ex;
            carry += total;
        }
        if (threadIdx.x == 0) tile_sum[t] = carry;
    }
}

__global__ void __launch_bounds__(256) k_scan_add(BoxDev b, const int4* tiles, int ntiles,
                                                   const int* tile_sum)
{
    if (!box_needs_rebuild(b)) return;
    __shared__ int s_off;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int4 tl = tiles[t];
        if (!rep_needs_rebuild(b, tl.x)) continue;
        if (threadIdx.x == 0) {
            int o = b.rep[tl.x].p_off;
            for (int u = tl.w; u < t; ++u) o += tile_sum[u];
            s_off = o;
        }
        __syncthreads();
        int o = s_off;
        for (int c = tl.y + (int)threadIdx.x; c < tl.z; c += blockDim.x) {
            int s = b.cell_start[c] + o;
            b.cell_start[c] = s;
            b.cell_end[c] = s;     // cursor for k_scatter; ends at start + count
            b.cell_count[c] = 0;   // ready for the next build
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_scatter: claim a slot inside the particle's new cell.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LJ_CHUNK) k_scatter(BoxDev b)
{
    if (!box_needs_rebuild(b)) return;
    const int tot = b.lw_coff[b.lw_hdr[0]];
    int kr = 0;
    for (int t = blockIdx.x; t < tot; t += gridDim.x) {
        int4 ch = b.chunk[work_chunk(b, t, kr)];
        int p = ch.y + (int)threadIdx.x;
        const bool act = p < ch.z;
        // warp-aggregated slot claims: one atomic per distinct cell of the
        // warp, each lane's slot = old cursor + its rank among the peers
        const int c = act ? b.cellB[p] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (act && lane == leader) base = atomicAdd(&b.cell_end[c], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (act) b.perm[base + __popc(peers & ((1u << lane) - 1u))] = p;
    }
}

// ---------------------------------------------------------------------------
// k_list_work: the work of a rebuild, one block.  The rebuilding replicas in
// order, with the prefixes of their cell and particle-chunk counts, so that
// the per-cell kernels (k_sortgather, k_nlist_lanes) and the per-chunk ones
// (k_bin, k_scatter, k_gather) stride over those cells and chunks only: a step
// in which a few replicas of many rebuild does not walk (and test) every cell
// and chunk of the batch.  Launched first in every rebuild sequence.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_list_work(BoxDev b)
{
    if (!box_needs_rebuild(b)) return;
    __shared__ int s_warp[33];
    int nsel = 0, ncell = 0, nch = 0;
    for (int base = 0; base < b.nrep; base += blockDim.x) {
        const int r = base + (int)threadIdx.x;
        const bool need = r < b.nrep && rep_needs_rebuild(b, r);
        int tsel, tcell, tch;
        const int xs = block_excl_scan(need ? 1 : 0, s_warp, tsel);
        const int xc = block_excl_scan(need ? b.rep[r].ncell : 0, s_warp, tcell);
        const int xh = block_excl_scan(need ? b.rep[r].nchunk : 0, s_warp, tch);
        if (need) {
            b.lw_rep[nsel + xs] = r;
            b.lw_off[nsel + xs] = ncell + xc;
            b.lw_coff[nsel + xs] = nch + xh;
        }
        nsel += tsel;
        ncell += tcell;
        nch += tch;
    }
    if (threadIdx.x == 0) {
        b.lw_off[nsel] = ncell;
        b.lw_coff[nsel] = nch;
        b.lw_hdr[0] = nsel;
    }
}

// ---------------------------------------------------------------------------
// k_sortgather: one warp per cell.  Order the members of the cell by their
// FP32 z offset from the cell centre (the value posq will hold), ties by
// user index (count of smaller keys; keys are unique), so the layout is a
// deterministic function of the positions and the list build can take, in
// every neighbour cell, the contiguous run of candidates within reach along
// z.  The alternative layout (order 1) sorts a cell by a space-filling curve
// over its 4 x 4 x 4 sub-cells first (Sec. 3: particles are sorted for
// locality); the list build then takes whole neighbour cells.  The ranks are
// written as each member's final slot (dst); k_gather then
// moves the state, the new cell-relative offsets (computed by k_bin) and
// their FP32 copy into the sorted arrays, one thread per particle.  (All
// pairs: one cell per replica, no order; k_sortgather gathers directly.)
// ---------------------------------------------------------------------------
// FP32 offset from the new cell centre, as posq will hold it (offB, from k_bin)
__device__ __forceinline__ float offB32(const BoxDev& b, int c, int p)
{
    if (b.prec == 0) return reinterpret_cast<const float*>(b.offB)[c * b.np + p];
    return __double2float_rn(b.offB[c * b.np + p]);
}

__device__ __forceinline__ unsigned long long sort_key(const BoxDev& b, const RepDev& R, int p)
{
    const float z = offB32(b, 2, p);
    const unsigned u = __float_as_uint(z);
    const unsigned ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // order-preserving
    if (b.order == 0) return ((unsigned long long)ord << 32) | (unsigned)b.uidB[p];
    // space-filling-curve order (Morton, or Z-order, curve over the cell's
    // 4 x 4 x 4 sub-cells: the sub-cell coordinates' bits interleaved), then
    // the z offset, then the user index (< 2^26) -- 6 + 32 + 26 bits
    unsigned m = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int sc = (int)floorf((offB32(b, c, p) / R.ellf[c] + 0.5f) * 4.f);
        sc = sc < 0 ? 0 : (sc > 3 ? 3 : sc);
        m |= (unsigned)(sc & 1) << c | (unsigned)(sc >> 1) << (c + 3);
    }
    return ((unsigned long long)m << 58) | ((unsigned long long)ord << 26) | (unsigned)b.uidB[p];
}

// Gather particle p (old order) into slot q of cell gc: its state, its new
// offsets (from k_bin) and their FP32 copy.  No arithmetic.
__device__ __forceinline__ void gather_one(const BoxDev& b, int p, int q, int gc)
{
    int ty = b.typeB[p];
    float of[3];
    for (int c = 0; c < 3; ++c) {
        b.xabs[c * b.np + q] = b.xabsB[c * b.np + p];
        if (b.prec == 0) {
            const float* ob = reinterpret_cast<const float*>(b.offB);
            float* ofs = reinterpret_cast<float*>(b.off);
            const float h = ob[c * b.np + p];
            ofs[c * b.np + q] = h;
            ofs[3 * b.np + c * b.np + q] = ob[3 * b.np + c * b.np + p];
            of[c] = h;
        } else {
            const double o = b.offB[c * b.np + p];
            b.off[c * b.np + q] = o;
            of[c] = __double2float_rn(o);
        }
        copy_acc(b, b.vel, b.velB, c, q, p);
        b.img[c * b.np + q] = b.imgB[c * b.np + p];
    }
    b.uid[q] = b.uidB[p];
    b.type[q] = ty;
    b.cell[q] = gc;
    float4 pq = make_float4(of[0], of[1], of[2], __int_as_float(ty));
    b.posq[q] = pq;
    b.ref[q] = pq;
}

__global__ void __launch_bounds__(256) k_sortgather(BoxDev b)
{
    if (!box_needs_rebuild(b)) return;
    if (b.all_pairs) {
        // one cell holds the whole replica and no list needs an order: a
        // particle's slot is its index inside the replica, one thread each
        const int tot = b.lw_coff[b.lw_hdr[0]];
        int kr = 0;
        for (int t = blockIdx.x; t < tot; t += gridDim.x) {
            const int4 ch = b.chunk[work_chunk(b, t, kr)];
            const RepDev& R = b.rep[ch.x];
            for (int s = ch.y + (int)threadIdx.x; s < ch.z; s += blockDim.x) {
                if (s == R.p_off) atomicAdd(&b.nbuild[ch.x], 1ull);   // a re-binning
                const int p = b.perm[s];
                gather_one(b, p, R.p_off + (b.uidB[p] - R.u_off), R.cell_off);
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int total = b.lw_off[b.lw_hdr[0]];
    int kr = 0;
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < total; t += gridDim.x * wpb) {
        const int gc = work_cell(b, t, kr);
        const RepDev& R = b.rep[b.lw_rep[kr]];
        int s0 = b.cell_start[gc];
        int n = b.cell_end[gc] - s0;
        for (int base = 0; base < n; base += 32) {
            int idx = base + lane;
            int p = idx < n ? b.perm[s0 + idx] : -1;
            const unsigned long long none = ~0ull;
            unsigned long long key = idx < n ? sort_key(b, R, p) : none;
            int rank = 0;
            for (int b2 = 0; b2 < n; b2 += 32) {
                unsigned long long k2 =
                    b2 == base ? key : ((b2 + lane < n) ? sort_key(b, R, b.perm[s0 + b2 + lane]) : none);
#pragma unroll 8
                for (int t = 0; t < 32; ++t) {
                    unsigned long long kt = __shfl_sync(0xffffffffu, k2, t);
                    rank += (kt < key) ? 1 : 0;
                }
            }
            if (idx < n) b.dst[s0 + idx] = s0 + rank;
        }
    }
}

__global__ void __launch_bounds__(LJ_CHUNK) k_gather(BoxDev b)
{
    if (b.all_pairs || !box_needs_rebuild(b)) return;
    const int tot = b.lw_coff[b.lw_hdr[0]];
    int kr = 0;
    for (int t = blockIdx.x; t < tot; t += gridDim.x) {
        const int4 ch = b.chunk[work_chunk(b, t, kr)];
        const int s = ch.y + (int)threadIdx.x;
        if (s >= ch.z) continue;
        const int p = b.perm[s];
        gather_one(b, p, b.dst[s], b.cellB[p]);
    }
}

// ---------------------------------------------------------------------------
// k_nlist: Verlet list of every particle of a rebuilding replica (Sec. 3),
// one segment per block.  The segment's tile (its 27-cell neighbourhood) is
// staged in shared memory and candidates are read from there.  Membership
// |d_ij|^2 < rl^2 is decided in FP32 from the cell-relative offsets; pairs
// within `band` of rl^2 are re-decided in FP64 from the wrapped positions
// with the minimum image, in the same operation order as the plain
// definition, so the lists equal the FP64 definition exactly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool exact_within(const BoxDev& b, const RepDev& R, int p, int j)
{
    double dd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d = __dsub_rn(b.xabs[c * b.np + p], b.xabs[c * b.np + j]);
        double t = rint(__ddiv_rn(d, R.L[c]));
        dd[c] = __dsub_rn(d, __dmul_rn(R.L[c], t));
    }
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])),
                          __dmul_rn(dd[2], dd[2]));
    return d2 < b.rl2;
}

__global__ void __launch_bounds__(LJ_LIST_THREADS, 3) k_nlist(BoxDev b)
{
    if (!box_needs_rebuild(b)) return;
    extern __shared__ __align__(16) float4 s_tile[];   // LJ_TILE_MAX entries
    __shared__ float4 s_shift[32];
    __shared__ int4 s_rng[LJ_SEG_MAX_CELLS * 27];   // (first, end, tile offset) per (cell, k)
    __shared__ int s_qoff[LJ_SEG_MAX_CELLS + 1];     // first quad of each cell
    __shared__ uint16_t s_flat[(LJ_LIST_THREADS / 32) * LJ_FLAT_MAX];   // per-warp candidate list
    __shared__ uint32_t s_kent[(LJ_LIST_THREADS / 32) * 32];             // per-warp entry bases
    __shared__ Tile s_t;
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_next;      // next quad of the segment to hand out
    __shared__ int s_longest;   // longest list this block built
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        s_longest = 0;
    }
    unsigned phase = 0;
    int cur_r = -1;
    const float lo2 = b.rl2f - b.band, hi2 = b.rl2f + b.band;
    for (int w = blockIdx.x; w < b.nseg; w += gridDim.x) {
        int4 sg = b.seg[w];
        int r = sg.x;
        if (!rep_needs_rebuild(b, r)) continue;   // block-uniform
        const RepDev& R = b.rep[r];
        __syncthreads();                          // previous segment done
        if (threadIdx.x < 32) {
            // warp 0: the tile's pieces, and the segment's quads per cell
            Tile t;
            seg_tile_warp(b, R, sg, t);
            const int lane = threadIdx.x;
            if (lane == 0) {
                s_t = t;
                if (w == R.seg_off) atomicAdd(&b.nbuild[r], 1ull);
            }
            const int cbase = R.cell_off + sg.y + R.nc[0] * sg.z;
            const int nqc = lane < sg.w ? (b.cell_end[cbase + lane] - b.cell_start[cbase + lane] + 3) >> 2 : 0;
            int incl = nqc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane < sg.w) s_qoff[lane] = incl - nqc;
            if (lane == sg.w - 1) s_qoff[sg.w] = incl;
            if (lane == 0) s_next = LJ_LIST_THREADS / 32;
        }
        if (r != cur_r && threadIdx.x < 32) {
            int k = threadIdx.x;
            s_shift[k] = k < 27 ? make_float4((float)(k % 3 - 1) * R.ellf[0], (float)((k / 3) % 3 - 1) * R.ellf[1],
                                              (float)(k / 9 - 1) * R.ellf[2], 0.f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cur_r = r;
        __syncthreads();
        const int n = s_t.n, p0 = s_t.p0;
        if (s_t.total > LJ_TILE_MAX) {
            if (threadIdx.x == 0) atomicOr(&b.err[0], LJ_ERRBIT_TILE);
            for (int il = threadIdx.x; il < n; il += blockDim.x) b.nbr_count[p0 + il] = 0;
            continue;
        }
        // neighbour-cell ranges of the segment's cells, with their tile offsets
        const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
        const int cy = sg.z % ny, cz = sg.z / ny;
        const int c0 = R.cell_off + sg.y + nx * sg.z;
        for (int idx = threadIdx.x; idx < sg.w * 27; idx += blockDim.x) {
            const int cl = idx / 27, k = idx % 27;
            const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
            const int cn = R.cell_off + wrapi(sg.y + cl + dx, nx) + nx * (wrapi(cy + dy, ny) + ny * wrapi(cz + dz, nz));
            const int js = b.cell_start[cn], je = b.cell_end[cn];
            int q = 2 * (3 * (dz + 1) + (dy + 1));
            if (!(js >= s_t.beg[q] && js < s_t.end[q])) ++q;
            s_rng[idx] = make_int4(js, je, s_t.base[q] - s_t.beg[q], 0);
        }
        if (s_t.total > 0 && !stage_tile_bulk(b.posq, s_t, s_tile, &s_bar, phase, b.err)) return;
        const float ell_h[3] = {0.5f * R.ellf[0], 0.5f * R.ellf[1], 0.5f * R.ellf[2]};
        const float rcull = b.rl2f + b.band;
        // reach along z of any pair the FP32 test can accept (r2 < rl^2 +
        // band implies dz^2 < rl^2 + band), with a margin for the rounding of
        // the shifted z values
        const float zreach = sqrtf(rcull) + 1e-3f;
        // work units: quads of particles of one cell (the quad's particles
        // share the cell, so their candidates are the same), handed out to
        // the warps one at a time as they finish (s_qoff, s_next set above)
        const int nquad = s_qoff[sg.w];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        uint16_t* flat = s_flat + warp * LJ_FLAT_MAX;
        uint32_t* kent = s_kent + warp * 32;
        for (int qd = warp; qd < nquad;) {
            int cl = 0;
            while (s_qoff[cl + 1] <= qd) ++cl;                  // warp-uniform
            const int cs = b.cell_start[c0 + cl], ce = b.cell_end[c0 + cl];
            const int p0q = cs + 4 * (qd - s_qoff[cl]);          // first particle of the quad
            const int nq = min(4, ce - p0q);                     // particles in the quad
            // the quad's particles, in every lane's registers
            float4 pq[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) pq[g] = b.posq[p0q + (g < nq ? g : 0)];
            const int4* rng = s_rng + cl * 27;
            // flatten the candidate cells (lane k owns stencil cell k); a cell
            // is dropped when its box lies beyond the list radius of all the
            // quad's particles
            int len = 0;
            int4 rk = make_int4(0, 0, 0, 0);
            if (lane < 27) {
                rk = rng[lane];
                const float4 sh = s_shift[lane];
                bool far = true;
                float zmin = pq[0].z, zmax = pq[0].z;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const float gx = fmaxf(fabsf(pq[g].x - sh.x) - ell_h[0], 0.f);
                    const float gy = fmaxf(fabsf(pq[g].y - sh.y) - ell_h[1], 0.f);
                    const float gz = fmaxf(fabsf(pq[g].z - sh.z) - ell_h[2], 0.f);
                    far = far && (g >= nq || gx * gx + gy * gy + gz * gz >= rcull);
                    zmin = fminf(zmin, pq[g].z);   // g >= nq repeats particle 0
                    zmax = fmaxf(zmax, pq[g].z);
                }
                if (!far && b.order != 0) {
                    len = rk.y - rk.x;   // space-filling-curve order: the whole cell
                } else if (!far) {
                    // the cell is sorted by z offset: keep the run with
                    // z_j + shift_z within zreach of the quad's z range
                    const float zlo = zmin - zreach - sh.z, zhi = zmax + zreach - sh.z;
                    const float* tz = reinterpret_cast<const float*>(s_tile) + 2;   // .z of tile entry t: tz[4 t]
                    int lo = rk.x + rk.z, hi = rk.y + rk.z;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (tz[4 * mid] < zlo) lo = mid + 1;
                        else hi = mid;
                    }
                    int e = rk.y + rk.z;
                    hi = e;
                    int lo2 = lo;
                    while (lo2 < hi) {
                        const int mid = (lo2 + hi) >> 1;
                        if (tz[4 * mid] <= zhi) lo2 = mid + 1;
                        else hi = mid;
                    }
                    rk.x = lo - rk.z;
                    rk.y = lo2 - rk.z;
                    len = rk.y - rk.x;
                }
            }
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            // entry of tile index t from cell k: t + kent[k] (the shift digits
            // above the slot, the slot being t minus the cell's tile offset)
            if (lane < 27) kent[lane] = entry_make(lane, 0) - (uint32_t)rk.z;
            const int self13 = p0q + __shfl_sync(0xffffffffu, rk.z, 13);   // tile index of the quad's first particle
            const int off = incl - len;
            int cnt[4] = {0, 0, 0, 0};
            bool nearb[4] = {false, false, false, false};   // saw a pair within the FP64 recheck band
            const unsigned lt_mask = (1u << lane) - 1u;
            uint32_t* const row0 = b.nbr + (size_t)b.K * p0q;   // list of the quad's first particle
            for (int w0 = 0; w0 < total; w0 += LJ_FLAT_MAX) {
                const int wn = min(total - w0, LJ_FLAT_MAX);
                __syncwarp();
                if (lane < 27) {
                    // lane k writes its cell's part of the window: (k, tile index)
                    const int ok = off - w0;
                    const int t_lo = max(0, -ok), t_hi = min(len, wn - ok);
                    const unsigned code = ((unsigned)lane << LJ_TILE_BITS) | (unsigned)(rk.x + rk.z);
                    for (int t = t_lo; t < t_hi; ++t) flat[ok + t] = (uint16_t)(code + (unsigned)t);
                }
                __syncwarp();
                // one candidate per lane, tested against the quad's particles;
                // pairs within the recheck band are kept here and settled in
                // FP64 afterwards
                // two candidates per lane per pass (t and t + 32): two
                // independent test-and-append chains for the scheduler
                for (int t0 = 0; t0 < wn; t0 += 64) {
                    float qx[2], qy[2], qz[2];
                    uint32_t ent[2];
                    int selfg[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = t0 + 32 * h + lane;
                        const unsigned e = t < wn ? flat[t] : 0u;
                        const int k = (int)(e >> LJ_TILE_BITS);
                        const int idx = (int)(e & LJ_TILE_MASK);
                        const float4 pj = s_tile[idx];
                        const float4 sh = s_shift[k];
                        // lanes past the window take a far point, whose r2 is inf
                        qx[h] = t < wn ? pj.x + sh.x : 1.0e38f;
                        qy[h] = pj.y + sh.y;
                        qz[h] = pj.z + sh.z;
                        ent[h] = (uint32_t)idx + kent[k];
                        // tile slices are disjoint, so the index alone finds the
                        // particle itself: quad slot idx - self13 (if in 0..3)
                        selfg[h] = idx - self13;
                    }
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (g >= nq) break;   // warp-uniform: slots past the quad's end take nothing
                        bool in[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float ddx = pq[g].x - qx[h], ddy = pq[g].y - qy[h], ddz = pq[g].z - qz[h];
                            const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            in[h] = r2 < hi2 && selfg[h] != g;
                            nearb[g] = nearb[g] || (in[h] && r2 >= lo2);
                        }
                        const unsigned b0 = __ballot_sync(0xffffffffu, in[0]);
                        const unsigned b1 = __ballot_sync(0xffffffffu, in[1]);
                        const int pos0 = cnt[g] + __popc(b0 & lt_mask);
                        const int pos1 = cnt[g] + __popc(b0) + __popc(b1 & lt_mask);
                        uint32_t* const rg = row0 + (size_t)b.K * g;
                        if (cnt[g] + 64 <= b.K) {   // warp-uniform: room for the whole pass
                            if (in[0]) rg[pos0] = ent[0];
                            if (in[1]) rg[pos1] = ent[1];
                        } else {                    // entries beyond the capacity are counted only
                            if (in[0] && pos0 < b.K) rg[pos0] = ent[0];
                            if (in[1] && pos1 < b.K) rg[pos1] = ent[1];
                        }
                        cnt[g] += __popc(b0) + __popc(b1);
                    }
                }
            }
            // FP64 decision for the particles that saw a pair near rl: drop the
            // band pairs beyond rl and compact their lists
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (g >= nq || !__any_sync(0xffffffffu, nearb[g])) continue;   // warp-uniform
                __syncwarp();   // the list's entries, stored by other lanes, are visible
                const int p = p0q + g;
                uint32_t* const row = row0 + (size_t)b.K * g;
                const int c = min(cnt[g], b.K);
                int kept = 0;
                for (int s0 = 0; s0 < c; s0 += 32) {
                    const int s = s0 + lane;
                    bool keep = false;
                    uint32_t ent = 0;
                    if (s < c) {
                        ent = row[s];
                        const int j = (int)(ent & LJ_IDX_MASK);
                        const int k = entry_k(ent);
                        const float4 pj = b.posq[j];
                        const float4 sh = s_shift[k];
                        const float ddx = pq[g].x - (pj.x + sh.x), ddy = pq[g].y - (pj.y + sh.y),
                                    ddz = pq[g].z - (pj.z + sh.z);
                        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        keep = r2 < lo2 || exact_within(b, R, p, j);
                    }
                    const unsigned bits = __ballot_sync(0xffffffffu, keep);
                    __syncwarp();
                    if (keep) row[kept + __popc(bits & lt_mask)] = ent;
                    kept += __popc(bits);
                }
                cnt[g] = cnt[g] - c + kept;   // entries beyond the capacity are counted, not stored
            }
            const int c = lane == 0 ? cnt[0] : lane == 1 ? cnt[1] : lane == 2 ? cnt[2] : cnt[3];
            if (lane < nq) {
                b.nbr_count[p0q + lane] = c;
                if (c > b.K) {
                    atomicOr(&b.err[0], LJ_ERRBIT_CAPACITY);
                    atomicMax(&b.err[1], c);
                }
            }
            const int cmax = __reduce_max_sync(0xffffffffu, lane < nq ? c : 0);
            int nxt = 0;
            if (lane == 0) {
                atomicMax(&s_longest, cmax);
                nxt = atomicAdd(&s_next, 1);
            }
            qd = __shfl_sync(0xffffffffu, nxt, 0);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_longest > 0) atomicMax(&b.err[2], s_longest);   // longest list of this build
}

// ---------------------------------------------------------------------------
// k_nlist_lanes: the same lists, one warp per cell and one lane per particle
// of the cell.  The warp streams the candidates of the 27 neighbour cells
// in chunks of 32: lane t loads candidate t of the chunk (coalesced, the
// next chunk's load in flight while this one is used), adds the cell's
// shift and drops it when its distance from the bounding box of the cell's
// particles is beyond the list radius (at least a quarter of the 27-cell
// block lies there); the kept
// candidates (shifted FP32 offset and a 16-bit code: neighbour cell k and
// index inside it) go to a per-warp ring in shared memory.  Every 32 staged
// candidates, each lane tests them all against its own particle -- one
// broadcast shared-memory load per candidate for the whole cell -- and
// appends the codes of its hits to its own row in shared memory (no
// ballots: every lane owns its row); at the end it writes the row out as
// list entries with 16-byte stores.  Pairs within `band` of rl^2 are
// re-decided in FP64 as in k_nlist (checked per batch of 32: the largest
// accepted r^2 tells whether any accepted pair lies in the band).  The x and
// y parts of d_ij and d_ij^2 are computed as FP32 pairs.
// ---------------------------------------------------------------------------
constexpr int kLaneWarps = LJ_LANE_THREADS / 32;
constexpr int kRing = 64;   // staged candidates per warp: < 32 waiting + one chunk
// Codes a lane holds in shared memory: fewer than 16 not yet written out plus
// one batch of 32.  Full 16-code blocks go out to the list before a batch
// that could overflow the buffer, so the rows' shared memory does not grow
// with the capacity K.
constexpr int kLaneRow = 48;

// r^2 of the pair (i, candidate q = o_j + shift) from n = -o_i.
__device__ __forceinline__ float lane_r2(const float2 nxy, float nz, const float4& q)
{
    const float2 d = __fadd2_rn(make_float2(q.x, q.y), nxy);
    const float dz = q.z + nz;
    const float2 s = __fmul2_rn(d, d);
    return fmaf(dz, dz, s.x + s.y);
}

__global__ void __launch_bounds__(LJ_LANE_THREADS, 8) k_nlist_lanes(BoxDev b)
{
    if (!box_needs_rebuild(b)) return;
    // row buffers, slot-major per warp: code e of lane l at [e][l] (the 32
    // lanes' stores of one step fall in distinct banks whatever their counts)
    extern __shared__ __align__(16) uint16_t s_rows[];   // per warp: kLaneRow x 32 codes
    __shared__ __align__(16) float s_cx[kLaneWarps][kRing];   // staged candidates: o_j + shift(k),
    __shared__ __align__(16) float s_cy[kLaneWarps][kRing];   // one array per component (four
    __shared__ __align__(16) float s_cz[kLaneWarps][kRing];   // candidates load as one 16-byte word)
    __shared__ __align__(16) uint32_t s_cc[kLaneWarps][kRing];   // and their codes
    __shared__ int2 s_rng[kLaneWarps][27];                // neighbour cell k: (first slot, end slot)
    __shared__ float4 s_sh[kLaneWarps][27];               // shift(k) = (dx, dy, dz) * cell edge
    __shared__ uint32_t s_base[kLaneWarps][32];           // entry of the first slot of cell k (27 used;
                                                          // stale codes past a row's end index up to 31)
    __shared__ int s_longest;
    if (threadIdx.x == 0) s_longest = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int K = b.K;
    uint16_t* const row = s_rows + (size_t)warp * kLaneRow * 32 + lane;   // slot e at row[32 e]
    float* const rx = s_cx[warp];
    float* const ry = s_cy[warp];
    float* const rz = s_cz[warp];
    uint32_t* const rc = s_cc[warp];
    const float lo2 = b.rl2f - b.band, hi2 = b.rl2f + b.band;
    const float rcull = hi2 + 1e-3f;   // staging margin for the rounding of the shifted offsets
    const float4* __restrict__ posq = b.posq;
    int longest = 0;
    const int nwarp = gridDim.x * kLaneWarps;
    const int total = b.lw_off[b.lw_hdr[0]];
    int kr = 0;
    for (int t = blockIdx.x * kLaneWarps + warp; t < total; t += nwarp) {
        const int gc = work_cell(b, t, kr);
        const int r = b.lw_rep[kr];
        const RepDev& R = b.rep[r];
        int cx, cy;
        const int cz = cell_coords(R, gc, cx, cy);
        const int cs = b.cell_start[gc], n = b.cell_end[gc] - cs;
        if (lane == 0 && gc == R.cell_off) atomicAdd(&b.nbuild[r], 1ull);
        __syncwarp();
        if (lane < 27) {
            const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            const int cn = R.cell_off + wrapi(cx + dx, R.nc[0]) +
                           R.nc[0] * (wrapi(cy + dy, R.nc[1]) + R.nc[1] * wrapi(cz + dz, R.nc[2]));
            const int js = b.cell_start[cn], je = b.cell_end[cn];
            s_rng[warp][lane] = make_int2(js, je);
            s_sh[warp][lane] = make_float4((float)dx * R.ellf[0], (float)dy * R.ellf[1], (float)dz * R.ellf[2], 0.f);
            s_base[warp][lane] = entry_make(lane, js);
            if (je - js > LJ_TILE_MAX) atomicOr(&b.err[0], LJ_ERRBIT_TILE);   // the 11-bit index: never at LJ densities
        }
        __syncwarp();
        for (int ib = 0; ib < n; ib += 32) {
            const bool act = ib + lane < n;
            const int i = cs + (act ? ib + lane : 0);
            float4 pi = posq[i];
            // the box of this pass's particles (tighter than the cell: the
            // candidates to test are those within the list radius of it)
            float lx = act ? pi.x : 1.0e30f, ly = act ? pi.y : 1.0e30f, lz = act ? pi.z : 1.0e30f;
            float ux = act ? pi.x : -1.0e30f, uy = act ? pi.y : -1.0e30f, uz = act ? pi.z : -1.0e30f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
                ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
                lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
                ux = fmaxf(ux, __shfl_xor_sync(0xffffffffu, ux, o));
                uy = fmaxf(uy, __shfl_xor_sync(0xffffffffu, uy, o));
                uz = fmaxf(uz, __shfl_xor_sync(0xffffffffu, uz, o));
            }
            if (!act) pi = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.f);   // a far point: r^2 is inf
            const float2 nxy = make_float2(-pi.x, -pi.y);
            const float nz = -pi.z;
            const uint32_t self = (13u << LJ_TILE_BITS) | (uint32_t)(ib + lane);   // the particle itself
            int cnt = 0;                   // codes in the row buffer
            int flushed = 0;               // list entries already written out (a multiple of 16)
            unsigned head = 0, tail = 0;   // ring positions (free-running; head stays a multiple of 32)
            uint4* const dst = reinterpret_cast<uint4*>(b.nbr + (size_t)K * i);   // the particle's row
            const uint32_t* const base = s_base[warp];
            // full 16-code blocks out to the list (the entry of cell k's first
            // slot + index), the rest to the buffer's front; entries past the
            // capacity are counted, not written
            auto flush = [&]() {
                const int nbk = act ? (cnt >> 4) : 0;
                for (int q = 0; q < nbk; ++q) {
                    if (flushed + 16 * (q + 1) <= K) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            uint32_t o[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const uint32_t h = row[32 * (16 * q + 4 * e + u)];
                                o[u] = base[h >> LJ_TILE_BITS] + (h & LJ_TILE_MASK);
                            }
                            dst[(flushed >> 2) + 4 * q + e] = make_uint4(o[0], o[1], o[2], o[3]);
                        }
                    }
                }
                const int rest = cnt - 16 * nbk;
                for (int q = 0; q < rest; ++q) row[32 * q] = row[32 * (16 * nbk + q)];
                flushed += 16 * nbk;
                cnt = rest;
                __syncwarp();
            };
            // test the staged candidates [head, head + cnt) against the lane's
            // particle and append the hits
            auto batch = [&](int nb) {
                const int c0 = cnt;
                const int h0 = (int)(head & (kRing - 1));
                float m = 0.f;   // largest accepted r^2 of the batch
                if (nb == 32) {   // the buffer has room for 32 more (flushed before the batch)
                    // branch-free, two candidates per step with FP32-pair
                    // arithmetic: every candidate's code is written to the
                    // next free slot (32-bit shared address), which advances
                    // only on a hit
                    uint32_t wa = (uint32_t)__cvta_generic_to_shared(row + 32 * cnt);
                    const float2 px = make_float2(nxy.x, nxy.x), py = make_float2(nxy.y, nxy.y),
                                 pz = make_float2(nz, nz);
                    // four candidates per step: one 16-byte broadcast load per
                    // component and for the codes
                    auto step2 = [&](float2 qx, float2 qy, float2 qz, uint32_t c0, uint32_t c1) {
                        const float2 dx = __fadd2_rn(qx, px), dy = __fadd2_rn(qy, py), dz = __fadd2_rn(qz, pz);
                        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                        const bool h1 = (r2.x < hi2) & (c0 != self);
                        asm volatile("st.shared.u16 [%0], %1;" ::"r"(wa), "h"((unsigned short)c0));
                        wa += h1 ? 64u : 0u;
                        m = fmaxf(m, h1 ? r2.x : 0.f);
                        const bool h2 = (r2.y < hi2) & (c1 != self);
                        asm volatile("st.shared.u16 [%0], %1;" ::"r"(wa), "h"((unsigned short)c1));
                        wa += h2 ? 64u : 0u;
                        m = fmaxf(m, h2 ? r2.y : 0.f);
                    };
#pragma unroll 2
                    for (int u = 0; u < 32; u += 4) {
                        const float4 qx = *reinterpret_cast<const float4*>(rx + h0 + u);
                        const float4 qy = *reinterpret_cast<const float4*>(ry + h0 + u);
                        const float4 qz = *reinterpret_cast<const float4*>(rz + h0 + u);
                        const uint4 cc = *reinterpret_cast<const uint4*>(rc + h0 + u);
                        step2(make_float2(qx.x, qx.y), make_float2(qy.x, qy.y), make_float2(qz.x, qz.y), cc.x, cc.y);
                        step2(make_float2(qx.z, qx.w), make_float2(qy.z, qy.w), make_float2(qz.z, qz.w), cc.z, cc.w);
                    }
                    asm volatile("" ::: "memory");   // the stores above stay above
                    __syncwarp();                      // and are seen by the reads below
                    cnt = (int)((wa - (uint32_t)__cvta_generic_to_shared(row)) >> 6);
                } else {
                    for (int u = 0; u < nb; ++u) {
                        const float4 q = make_float4(rx[h0 + u], ry[h0 + u], rz[h0 + u], 0.f);
                        const float r2 = lane_r2(nxy, nz, q);
                        const uint32_t code = rc[h0 + u];
                        if (r2 < hi2 && code != self) {
                            row[32 * cnt] = (uint16_t)code;
                            ++cnt;
                            m = fmaxf(m, r2);
                        }
                    }
                }
                // FP64 decision of the batch's accepted pairs near rl (rare)
                if (__any_sync(0xffffffffu, m >= lo2) && m >= lo2) {
                    int w = c0;
                    const int e = cnt;
                    for (int q = c0; q < e; ++q) {
                        const uint32_t code = row[32 * q];
                        const int k = (int)(code >> LJ_TILE_BITS);
                        const int j = (int)(s_base[warp][k] & LJ_IDX_MASK) + (int)(code & LJ_TILE_MASK);
                        const float4 pj = posq[j];
                        const float4 sh = s_sh[warp][k];
                        const float4 qj = make_float4(pj.x + sh.x, pj.y + sh.y, pj.z + sh.z, 0.f);
                        if (lane_r2(nxy, nz, qj) < lo2 || exact_within(b, R, i, j)) row[32 * w++] = (uint16_t)code;
                    }
                    cnt = w;
                }
                head += 32u;
            };
            // chunk iterator over the neighbour cells: (k, j0), 32 slots at a time
            int k = 0, j0 = s_rng[warp][0].x;
            while (k < 27 && j0 >= s_rng[warp][k].y) {
                ++k;
                if (k < 27) j0 = s_rng[warp][k].x;
            }
            float4 raw = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < 27 && j0 + lane < s_rng[warp][k].y) raw = posq[j0 + lane];
            while (k < 27) {
                const int kc = k, len = min(32, s_rng[warp][k].y - j0);
                const int ic = j0 - s_rng[warp][k].x + lane;   // index of this lane's candidate in cell kc
                const float4 cur = raw;
                j0 += 32;
                while (k < 27 && j0 >= s_rng[warp][k].y) {
                    ++k;
                    if (k < 27) j0 = s_rng[warp][k].x;
                }
                if (k < 27 && j0 + lane < s_rng[warp][k].y) raw = posq[j0 + lane];   // next chunk, in flight
                // stage: shift into the cell's frame, keep what can be within reach of the cell
                const float4 sh = s_sh[warp][kc];
                const float qx = cur.x + sh.x, qy = cur.y + sh.y, qz = cur.z + sh.z;
                const float gx = fmaxf(fmaxf(lx - qx, qx - ux), 0.f), gy = fmaxf(fmaxf(ly - qy, qy - uy), 0.f),
                            gz = fmaxf(fmaxf(lz - qz, qz - uz), 0.f);
                const bool keep = lane < len && fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < rcull;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int t = (int)((tail + __popc(bal & lt)) & (kRing - 1));
                    rx[t] = qx;
                    ry[t] = qy;
                    rz[t] = qz;
                    rc[t] = ((uint32_t)kc << LJ_TILE_BITS) | (uint32_t)ic;
                }
                tail += __popc(bal);
                __syncwarp();
                if (tail - head >= 32) {
                    if (__any_sync(0xffffffffu, cnt > kLaneRow - 32)) flush();
                    batch(32);
                }
                __syncwarp();
            }
            if (tail > head) {
                if (__any_sync(0xffffffffu, cnt > kLaneRow - 32)) flush();
                batch((int)(tail - head));
            }
            __syncwarp();
            const int c = flushed + cnt;
            if (act) {
                // the buffer's codes -> list entries, 4 at a time, up to the capacity
                const int cst = min(cnt, K - flushed);
                for (int e = 0; 4 * e < cst; ++e) {   // rows end inside a block: masked by the count
                    uint32_t o[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t h = row[32 * (4 * e + u)];
                        o[u] = base[h >> LJ_TILE_BITS] + (h & LJ_TILE_MASK);
                    }
                    dst[(flushed >> 2) + e] = make_uint4(o[0], o[1], o[2], o[3]);
                }
                b.nbr_count[i] = c;
                if (c > K) {
                    atomicOr(&b.err[0], LJ_ERRBIT_CAPACITY);
                    atomicMax(&b.err[1], c);
                }
                longest = max(longest, c);
            }
            __syncwarp();
        }
    }
    longest = __reduce_max_sync(0xffffffffu, longest);
    if (lane == 0 && longest > 0) atomicMax(&s_longest, longest);
    __syncthreads();
    if (threadIdx.x == 0 && s_longest > 0) atomicMax(&b.err[2], s_longest);
}

// Condition of the step graph's list-update node: 1 when the integrator (or
// the host) raised the box-wide rebuild word, so that steps without a build
// launch none of the rebuild kernels; each 1 is counted (launch accounting).
__global__ void k_set_rebuild_cond(cudaGraphConditionalHandle h, const int* any_req, unsigned long long* runs)
{
    const bool go = *((volatile const int*)any_req) != 0;
    if (go) atomicAdd(runs, 1ull);
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

}  // namespace

cudaError_t launch_set_rebuild_cond(cudaGraphConditionalHandle h, const BoxDev& b, unsigned long long* runs,
                                    cudaStream_t s)
{
    k_set_rebuild_cond<<<1, 1, 0, s>>>(h, b.any_req, runs);
    return cudaGetLastError();
}

cudaError_t launch_bin(const BoxDev& b, int from_abs, Launch l)
{
    k_bin<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, from_abs);
    return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const BoxDev& b, const int4* tiles, int ntiles, int* tile_sum,
                              Launch l)
{
    k_scan_tiles<<<l.grid, 1024, 0, l.s>>>(b, tiles, ntiles, tile_sum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_add<<<l.grid, 256, 0, l.s>>>(b, tiles, ntiles, tile_sum);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const BoxDev& b, Launch l)
{
    k_scatter<<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_sortgather(const BoxDev& b, Launch l, Launch lg)
{
    k_sortgather<<<l.grid, 256, 0, l.s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || b.all_pairs) return e;
    k_gather<<<lg.grid, LJ_CHUNK, 0, lg.s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_nlist(const BoxDev& b, Launch l)
{
    const int dyn = LJ_TILE_MAX * 16;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_nlist, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_nlist<<<l.grid, LJ_LIST_THREADS, dyn, l.s>>>(b);
    return cudaGetLastError();
}

// Shared memory of k_nlist_lanes (any capacity K): kLaneRow 16-bit code
// slots per lane.
size_t nlist_lanes_smem(int) { return (size_t)LJ_LANE_THREADS * (size_t)kLaneRow * 2u; }

cudaError_t launch_list_work(const BoxDev& b, cudaStream_t s)
{
    k_list_work<<<1, 1024, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_nlist_lanes(const BoxDev& b, Launch l)
{
    static size_t attr = 0;
    const size_t dyn = nlist_lanes_smem(b.K);
    if (dyn > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_nlist_lanes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        attr = dyn;
    }
    k_nlist_lanes<<<l.grid, LJ_LANE_THREADS, dyn, l.s>>>(b);
    return cudaGetLastError();
}

int ljmd_scan_tile_cells() { return kScanTile; }
