// ljmd_internal.cuh -- device data layout and kernel launchers of libljmd.
//
// Layout in HBM (one batch of nrep replicas, np particle slots):
//   * particles of replica r occupy slots [p_off, p_off + n) with p_off a
//     multiple of 32; slots are sorted by (cell, FP32 z offset, user index)
//     at every list build (particle binning, Sec. 3 "Code structure").
//   * the integrator state of a particle is its cell id plus the offset from
//     that cell's centre ("cell-relative offset"), so FP32 copies of the
//     offsets keep ~1e-7 absolute resolution whatever the box size.  In
//     MD_PREC_MIXED_DS the offsets and velocities are double-single pairs
//     (hi, lo) of FP32; otherwise FP64.
//   * posq[p] = (float offset x, y, z, type bits) feeds the FP32 pair kernels.
//   * pair work is done per "segment": a run of up to S consecutive cells
//     along x inside one row (cy, cz) of a replica.  Its particles are one
//     contiguous slot range, and the 27-cell neighbourhood of all its cells
//     is the "tile": 9 rows x (S + 2) cells, i.e. at most 18 contiguous slot
//     ranges ("pieces"), staged in shared memory.
//   * Verlet lists (Sec. 3) are 32-bit entries: the image shift of j's cell
//     relative to i's cell as three 2-bit digits (dz+1, dy+1, dx+1 in bits
//     31-30, 29-28, 27-26) and the slot j in bits 25-0, so
//     d_ij = (o_i - o_j) - (dx, dy, dz) * cell edge, decoded with integer and
//     FP32 arithmetic (no table).  The stencil code k = 9(dz+1) + 3(dy+1) +
//     (dx+1) orders the 27 cells.
//     Entry s of particle p is nbr[p K + s] (K a multiple of 16): the FP32
//     force kernel reads a row in blocks of 16 entries, one 16-byte load per
//     thread of the particle; entries past the count are never written, and
//     the kernel replaces them by the sentinel slot np in the last block.
//   * the list build works per segment with the tile staged in shared memory;
//     the pair-force kernels work per 128-particle chunk, 4 threads per
//     particle, and gather neighbour offsets through L1 (the 64 particles of a
//     block pass are consecutive, so they share one 27-cell neighbourhood).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define LJ_MAXT 8
#define LJ_IDX_BITS 26         // slot indices must stay below 2^26
#define LJ_IDX_MASK ((1u << LJ_IDX_BITS) - 1u)
#define LJ_TILE_BITS 11
#define LJ_TILE_MAX (1 << LJ_TILE_BITS)
#define LJ_TILE_MASK (LJ_TILE_MAX - 1)
#define LJ_CHUNK 128           // particles per work item (one CTA pass)
#define LJ_FORCE_THREADS 256   // threads of the FP32 pair-force kernel
#define LJ_FORCE_WARPS (LJ_FORCE_THREADS / 32)   // its (E_pot, W) shares per chunk
#define LJ_KIN_WARPS (LJ_CHUNK / 32)   // E_kin shares per chunk (one per warp of the integrator)
#define LJ_THERMO_THREADS 256  // threads of the energy reduction
#define LJ_THERMO_CHUNKS 256   // chunks of one energy-reduction item
#define LJ_LIST_THREADS 256    // threads of the list-build kernel
#define LJ_LANE_THREADS 128    // threads of the lane-per-particle list-build kernel
#define LJ_F64_THREADS 128     // threads of the FP64 pair kernel (one per particle)
#define LJ_F64_WARPS (LJ_F64_THREADS / 32)   // its (E_pot, W) shares per chunk
#define LJ_TPP 4               // threads per particle in the pair kernels
#define LJ_SEG_MAX_CELLS 16    // most cells in one segment
#define LJ_FLAT_MAX 1024       // candidates of one cell's 27-cell neighbourhood (list build)
#define LJ_LIST_SMEM (32 * 1024)   // bytes of a segment's list staged in smem
#define LJ_ROW_BLOCK 16        // the FP32 force kernel reads list rows in blocks of this many entries
#define LJ_BRICK_THREADS 256   // threads of the tiled FP32 pair-force kernel (LJ_TPP per particle)
#define LJ_BRICK_WARPS (LJ_BRICK_THREADS / 32)   // its (E_pot, W) shares per brick
#define LJ_BRICK_TILE 2048     // particles of a brick's neighbourhood staged in shared memory
// In a row's last block the FP32 force kernel replaces the entries past the
// count by slot np, one past the last particle: posq[np] holds this offset on
// every axis, so that the pair distance, squared, stays finite (~3e30) and
// far beyond any cutoff.
#define LJ_SENTINEL_OFF 1.0e15f

// error word bits (err[0]); err[1] = largest list length beyond capacity;
// err[2] = longest list of the last builds
#define LJ_ERRBIT_CAPACITY 1
#define LJ_ERRBIT_NONFINITE 2
#define LJ_ERRBIT_TIMEOUT 4
#define LJ_ERRBIT_TILE 8       // a tile exceeded LJ_TILE_MAX particles

// integrate kernel modes
#define LJ_STEP_FIRST 0        // half kick + drift
#define LJ_STEP_MID 1          // finalize previous step + half kick + drift
#define LJ_STEP_LAST 2         // finalize

struct RepDev {
    double L[3];
    double wrap_hi[3];         // L (1 - 2^-50): 0 <= x < wrap_hi implies floor(x / L) = 0
    double ell[3];             // cell edge lengths
    double inv_ell[3];
    float ellf[3];
    float ell_lo[3];           // ell - ellf: (ellf, ell_lo) is the edge as a double-single pair
    int nc[3];
    int cell_off, ncell;
    int p_off, n;              // first slot, real particles
    int u_off;                 // first user index
    int chunk_off, nchunk;     // particle work items of this replica
    int ti_off, nti;           // energy-reduction items of this replica
    int seg_off, nseg;         // segments of this replica
    int S;                     // cells per segment (along x)
    int br[3];                 // brick edge in cells (1 or 2) of the tiled force kernel
    int brick_off, nbrick;     // its bricks of this replica
};

// Slot ranges of a segment's tile: piece q (0..17) is row rr = q/2 with
// rr = 3(dz+1) + (dy+1); tile index of slot j in piece q = base[q] + j - beg[q].
struct Tile {
    int beg[18];
    int end[18];
    int base[18];
    int total;
    int p0, n;                 // the segment's own particles
};

// pair parameters, FP32 and FP64 copies: per type pair (a*nt+b)
struct LJDev {
    int nt;
    int shift_on;
    // FP32 lj1/lj2 form: f = r2i r6i (c12 r6i - c6), u = r6i (e12 r6i - e6) - shift
    float c12[LJ_MAXT * LJ_MAXT], c6[LJ_MAXT * LJ_MAXT], e12[LJ_MAXT * LJ_MAXT], e6[LJ_MAXT * LJ_MAXT];
    // Hessian and parameter-derivative coefficients (adjoint):
    // A = r2i^2 r6i (a12 r6i - a6); dF/dsigma coefficient r2i r6i (g12 r6i - g6)
    float a12[LJ_MAXT * LJ_MAXT], a6[LJ_MAXT * LJ_MAXT], g12[LJ_MAXT * LJ_MAXT], g6[LJ_MAXT * LJ_MAXT];
    float inv_eps[LJ_MAXT * LJ_MAXT];
    float sig2[LJ_MAXT * LJ_MAXT], eps48[LJ_MAXT * LJ_MAXT], eps4[LJ_MAXT * LJ_MAXT];
    float rc2[LJ_MAXT * LJ_MAXT], shift[LJ_MAXT * LJ_MAXT];
    double dsig2[LJ_MAXT * LJ_MAXT], deps48[LJ_MAXT * LJ_MAXT], deps4[LJ_MAXT * LJ_MAXT];
    double drc2[LJ_MAXT * LJ_MAXT], dshift[LJ_MAXT * LJ_MAXT];
    double deps[LJ_MAXT * LJ_MAXT], dsig[LJ_MAXT * LJ_MAXT];
};

// Everything a kernel needs, passed by value.
struct BoxDev {
    int nrep, np, nchunk, ncell;
    int K;                     // list capacity (slots per particle; a multiple of LJ_ROW_BLOCK)
    int prec;                  // md_precision
    int nt;                    // species count
    float disp_thr2;           // rebuild when |displacement|^2 > this (FP32)
    float band;                // FP64 recheck band on |d|^2 around rl^2
    float rl2f;
    // one species (nt == 1): its FP32 pair constants, read by the force
    // kernel from the kernel parameters (no registers held for them)
    float4 c1;                 // c12, c6, e12, e6
    float rc2_1, esh_1;
    float3 ell1;               // one replica (nrep == 1): its cell edge, FP32
    double rl2;
    const RepDev* rep;
    const int4* chunk;         // (rep, p_begin, p_end, chunk index)
    const int4* titem;         // energy reduction: (rep, first chunk, end chunk, 0)
    int ntitem;
    const int4* seg;           // (rep, first cell x, row = cy + ny cz, cells)
    int nseg;
    const LJDev* lj;
    // particle arrays (sorted order)
    float4* posq;              // np + 1 entries: the last is the sentinel (LJ_SENTINEL_OFF)
    float4* ref;
    double* off;               // FP64: off[c*np + p]; DS: float hi[c*np+p], lo[3np + c*np + p]
    double* vel;               // same layout as off
    int* img;                  // img[c*np + p]
    int* uid;
    int* type;
    int* cell;
    double* xabs;              // xabs[c*np + p]: positions of the last build
    float4* force4;            // FP32 forces (mixed modes)
    double* force64;           // FP64 forces (FP64 mode), force64[c*np + p]
    // old-order copies during a rebuild
    double* xabsB;
    double* offB;              // new offsets from the new cell centre (layout of `off`), from k_bin
    // work of a rebuild: the rebuilding replicas in order (lw_rep[0 .. lw_hdr[0])),
    // the first index of each one's cells (lw_off) and particle chunks (lw_coff)
    // in their concatenations (one more entry each: the totals); written by
    // k_list_work at the head of a rebuild
    int* lw_hdr;
    int* lw_rep;
    int* lw_off;
    int* lw_coff;
    double* velB;
    int* imgB;
    int* uidB;
    int* typeB;
    int* cellB;
    int* perm;                 // slot -> old index, during a rebuild
    int* dst;                  // slot of perm -> final slot (ranked in its cell), during a rebuild
    // cells
    int* cell_count;
    int* cell_start;
    int* cell_end;
    const int* cell_rep;
    // lists
    uint32_t* nbr;
    int* nbr_count;
    // per-replica control
    unsigned* disp_max;        // FP32 bits of the largest |displacement|^2
    int* rebuild_req;          // host-forced rebuild
    int* any_req;              // nonzero when some replica may need a build
    unsigned long long* nbuild;
    int* err;
    // Andersen-like thermostat: a particle collides when word 0 of its Philox
    // draw is below tstat_thr (0: off); the bath temperature is per replica
    unsigned tstat_thr;
    unsigned long long tstat_seed;
    const double* tstat_T;
    long long* step_ctr;       // steps since md_set_thermostat (device word)
    int all_pairs;             // every cutoff infinite: forces over all pairs, no lists
    int force_tiles;           // FP32 list forces by the tiled kernel (k_force_tile_f32)
    const int4* brick;         // its work items: (replica, first cell x, y, z) of bricks of up to
    int nbrick;                // rep.br[0] x br[1] x br[2] cells
    int order;                 // order inside a cell: 0 z runs (LJ_ORDER_ZRUN), 1 Morton sub-cells
    int ap_js;                 // all pairs: slices of the j range per chunk
    float4* ap_part;           // [slice][slot] partial FP32 forces
    double* ap_part64;         // [slice][3][slot] partial FP64 forces
    double* ap_pe;             // [chunk * ap_js + slice][2] partial E_pot, W
    unsigned* ap_cnt;          // per chunk: slices done (the last one resets)
    // per-chunk FP64 partial sums
    double* part_f;            // [(chunk*pf_stride + q)*2 + 0] = E_pot share, [+1] = W share
    int pf_stride;             // (E_pot, W) shares per chunk: one per warp of the list kernels, 1 for all pairs
    int pf_ds;                 // 1: each share is a double-single pair (hi, lo floats in the double's
                               // 8 bytes: the FP32 list kernels), 0: a double; the tiled kernel
                               // leaves pf_stride shares per brick instead of per chunk
    double* part_k;            // [chunk*LJ_KIN_WARPS + warp] = E_kin share
    double* part_t;            // [item*3 + 0..2] = E_pot, W, E_kin of a reduction item
    unsigned* tcount;          // per replica: reduction items finished (last one resets)
};

// ---- double-single helpers (Dekker / Knuth error-free transformations) ----
__device__ __forceinline__ void ds_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ds_fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (h, l) += x  (x a single float)
__device__ __forceinline__ void ds_add_f(float& h, float& l, float x)
{
    float s, e;
    ds_two_sum(h, x, s, e);
    e = __fadd_rn(e, l);
    ds_fast_two_sum(s, e, h, l);
}
// (h, l) += (xh, xl)
__device__ __forceinline__ void ds_add_ds(float& h, float& l, float xh, float xl)
{
    float s, e;
    ds_two_sum(h, xh, s, e);
    e = __fadd_rn(e, __fadd_rn(l, xl));
    ds_fast_two_sum(s, e, h, l);
}
// (ph, pl) = (ah, al) * (bh, bl), dropping al*bl
__device__ __forceinline__ void ds_mul_ds(float ah, float al, float bh, float bl, float& ph,
                                          float& pl)
{
    float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    ds_fast_two_sum(p, e, ph, pl);
}
__device__ __forceinline__ void ds_from_double(double x, float& h, float& l)
{
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Sum over the warp in double-single arithmetic (FP32 pairs, Knuth's
// two-sum at every step), returned as FP64 in every lane: an FP64-class sum
// on the FP32 pipe (FP64 adds are scarce on this GPU).  The butterfly order
// is fixed, so the result is deterministic.
__device__ __forceinline__ float2 warp_sum_ds2(float x)
{
    float h = x, l = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        ds_add_ds(h, l, oh, ol);
    }
    return make_float2(h, l);
}
__device__ __forceinline__ double warp_sum_ds(float x)
{
    const float2 s = warp_sum_ds2(x);
    return (double)s.x + (double)s.y;
}

// Cheap block-level early exit of the rebuild kernels: nothing to do unless
// the integrator or the host raised the box-wide request word.
__device__ __forceinline__ bool box_needs_rebuild(const BoxDev& b)
{
    return *((volatile const int*)b.any_req) != 0;
}

__device__ __forceinline__ bool rep_needs_rebuild(const BoxDev& b, int r)
{
    return b.rebuild_req[r] != 0 || __uint_as_float(b.disp_max[r]) > b.disp_thr2;
}

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// 1/x by the hardware reciprocal (PTX rcp.approx.ftz.f32: one special-function
// instruction, relative error within 2^-23 for normal x); the pair kernels
// pass r^2 > 0 and finite.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- list entries ----
__host__ __device__ __forceinline__ uint32_t entry_make(int k, int j)
{
    return ((uint32_t)(k / 9) << 30) | ((uint32_t)((k / 3) % 3) << 28) | ((uint32_t)(k % 3) << 26) |
           (uint32_t)j;
}
__device__ __forceinline__ int entry_k(uint32_t e)
{
    return 9 * (int)(e >> 30) + 3 * (int)((e >> 28) & 3u) + (int)((e >> 26) & 3u);
}
// The digit at bit `pos` minus one, as an exact FP32 value in {-1, 0, 1}:
// 0x4B400000 is 1.5 * 2^23, whose mantissa's low bits take the digit.
__device__ __forceinline__ float entry_unit(uint32_t e, int pos)
{
    return __uint_as_float(0x4B400000u | ((e >> pos) & 3u)) - 12582913.0f;
}

// ---- Philox4x32-10 (Salmon et al., SC'11), counter-based random numbers ----
// Ten rounds: words 0 and 2 are multiplied by two odd constants; the high
// halves, crossed and mixed with words 1, 3 and the key, and the low halves
// form the next counter; the key advances by two Weyl constants per round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ---- bulk asynchronous copies (TMA, non-tensor) into shared memory ----
// One thread arms an mbarrier with the byte count and issues one
// cp.async.bulk per contiguous piece; every thread then waits on the
// barrier's phase.  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arm(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Order earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Wait for phase `parity` of the barrier; gives up after a bounded number of
// polls (returns false; the caller records LJ_ERRBIT_TIMEOUT and stops).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity)
{
    unsigned a = smem_u32(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Stage the FP32 offsets of a tile (and, if list_bytes > 0, a contiguous
// list block) into shared memory with bulk copies
// (thread 0 issues; all threads wait).  Returns false, for every thread of
// the block alike, on a timed-out wait.  Must be called by all threads.
__device__ __forceinline__ bool stage_tile_bulk(const float4* posq, const Tile& t, float4* s_tile,
                                                unsigned long long* bar, unsigned& phase, int* err,
                                                void* s_list = nullptr, const void* g_list = nullptr,
                                                unsigned list_bytes = 0)
{
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        unsigned bytes = (unsigned)t.total * 16u + list_bytes;
        mbar_arm(bar, bytes);
        for (int q = 0; q < 18; ++q) {
            int len = t.end[q] - t.beg[q];
            if (len > 0) bulk_g2s(s_tile + t.base[q], posq + t.beg[q], (unsigned)len * 16u, bar);
        }
        if (list_bytes) bulk_g2s(s_list, g_list, list_bytes, bar);
    }
    bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;   // one decision for the whole block
    if (!ok && threadIdx.x == 0) atomicOr(err, LJ_ERRBIT_TIMEOUT);
    return ok;
}

// Slot ranges of segment sg's tile (any thread may compute it).
__device__ __forceinline__ void seg_tile(const BoxDev& b, const RepDev& R, int4 sg, Tile& t)
{
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const int cx0 = sg.y, cy = sg.z % ny, cz = sg.z / ny, S = sg.w;
    int acc = 0;
    for (int rr = 0; rr < 9; ++rr) {
        int dy = rr % 3 - 1, dz = rr / 3 - 1;
        int rowc = R.cell_off + nx * (wrapi(cy + dy, ny) + ny * wrapi(cz + dz, nz));
        int a0, a1, b0 = 0, b1 = -1;   // cell x ranges of the two pieces (inclusive)
        if (S + 2 >= nx) {
            a0 = 0;
            a1 = nx - 1;
        } else if (cx0 - 1 < 0) {
            a0 = nx - 1; a1 = nx - 1; b0 = 0; b1 = cx0 + S;
        } else if (cx0 + S >= nx) {
            a0 = cx0 - 1; a1 = nx - 1; b0 = 0; b1 = cx0 + S - nx;
        } else {
            a0 = cx0 - 1; a1 = cx0 + S;
        }
        int q = 2 * rr;
        t.beg[q] = b.cell_start[rowc + a0];
        t.end[q] = b.cell_end[rowc + a1];
        t.base[q] = acc;
        acc += t.end[q] - t.beg[q];
        if (b1 >= b0) {
            t.beg[q + 1] = b.cell_start[rowc + b0];
            t.end[q + 1] = b.cell_end[rowc + b1];
        } else {
            t.beg[q + 1] = t.end[q + 1] = 0;
        }
        t.base[q + 1] = acc;
        acc += t.end[q + 1] - t.beg[q + 1];
    }
    t.total = acc;
    int c0 = R.cell_off + cx0 + nx * sg.z;
    t.p0 = b.cell_start[c0];
    t.n = b.cell_end[c0 + S - 1] - t.p0;
}

// The same tile computed by one warp (all 32 lanes call it): lane q < 18
// loads the bounds of piece q, the bases are an exclusive prefix over the
// pieces.  Returns the tile in every lane's t (lane 0 may store it).
__device__ __forceinline__ void seg_tile_warp(const BoxDev& b, const RepDev& R, int4 sg, Tile& t)
{
    const int lane = threadIdx.x & 31;
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const int cx0 = sg.y, cy = sg.z % ny, cz = sg.z / ny, S = sg.w;
    int beg = 0, end = 0;
    if (lane < 18) {
        const int rr = lane >> 1, half = lane & 1;
        const int dy = rr % 3 - 1, dz = rr / 3 - 1;
        const int rowc = R.cell_off + nx * (wrapi(cy + dy, ny) + ny * wrapi(cz + dz, nz));
        int a0, a1, b0 = 0, b1 = -1;   // cell x ranges of the row's two pieces (inclusive)
        if (S + 2 >= nx) {
            a0 = 0;
            a1 = nx - 1;
        } else if (cx0 - 1 < 0) {
            a0 = nx - 1; a1 = nx - 1; b0 = 0; b1 = cx0 + S;
        } else if (cx0 + S >= nx) {
            a0 = cx0 - 1; a1 = nx - 1; b0 = 0; b1 = cx0 + S - nx;
        } else {
            a0 = cx0 - 1; a1 = cx0 + S;
        }
        if (half == 0) {
            beg = b.cell_start[rowc + a0];
            end = b.cell_end[rowc + a1];
        } else if (b1 >= b0) {
            beg = b.cell_start[rowc + b0];
            end = b.cell_end[rowc + b1];
        }
    }
    const int len = end - beg;
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        t.beg[q] = __shfl_sync(0xffffffffu, beg, q);
        t.end[q] = __shfl_sync(0xffffffffu, end, q);
        t.base[q] = __shfl_sync(0xffffffffu, incl - len, q);
    }
    t.total = __shfl_sync(0xffffffffu, incl, 17);
    const int c0 = R.cell_off + cx0 + nx * sg.z;
    t.p0 = b.cell_start[c0];
    t.n = b.cell_end[c0 + S - 1] - t.p0;
}

// ---- launchers (defined in the kernel translation units) ----
struct Launch {
    int grid;
    int block;
    cudaStream_t s;
};

// k_rebuild.cu
cudaError_t launch_bin(const BoxDev& b, int from_abs, Launch l);
cudaError_t launch_scan_tiles(const BoxDev& b, const int4* tiles, int ntiles, int* tile_sum,
                              Launch l);
int ljmd_scan_tile_cells();
cudaError_t launch_scatter(const BoxDev& b, Launch l);
cudaError_t launch_sortgather(const BoxDev& b, Launch l, Launch lg);   // rank (l), then gather (lg) unless all pairs
cudaError_t launch_nlist(const BoxDev& b, Launch l);
// one warp per cell, one lane per particle (rows staged in shared memory:
// nlist_lanes_smem(K) bytes per block)
cudaError_t launch_nlist_lanes(const BoxDev& b, Launch l);
cudaError_t launch_list_work(const BoxDev& b, cudaStream_t s);   // one block; before the cell kernels
size_t nlist_lanes_smem(int K);
// sets a step graph's IF-node condition from the box-wide rebuild word
cudaError_t launch_set_rebuild_cond(cudaGraphConditionalHandle h, const BoxDev& b, unsigned long long* runs,
                                    cudaStream_t s);

// k_force.cu
cudaError_t launch_force(const BoxDev& b, int energy, Launch l);
cudaError_t launch_thermo(const BoxDev& b, double* out, int with_kin, Launch l);
int force_tile_blocks_per_sm(int mono);   // resident blocks of the tiled force kernel

// k_adjoint.cu
cudaError_t launch_adj_pre(const BoxDev& b, double* lx, double* lv, const double* g, float4* u_slot, double h,
                           int pre, Launch l);
// HVP of u at the state of b, g <- H u, lx <- lx - h/2 g (when upd), and
// part_g += *weight * the state's parameter-gradient shares
cudaError_t launch_hvp(const BoxDev& b, const float4* u_slot, double* lx, double* g, double h, int upd,
                       const double* weight, double* part_g, Launch l);
cudaError_t launch_param_reduce(const double* part_g, int nchunk, int twoP, const double* weight,
                                double* theta_grad, cudaStream_t s);
cudaError_t launch_pair_hist(const BoxDev& b, int nbins, double rhist, double width, double rmax, double* part_h,
                             double* h, Launch l);
cudaError_t launch_pair_hist_grad(const BoxDev& b, int nbins, double rhist, double width, double rmax,
                                  const double* coef, double* grad, Launch l);

// k_integrate.cu
cudaError_t launch_integrate(const BoxDev& b, int mode, int energy, double dt, int sidx, Launch l);
cudaError_t launch_step_advance(long long* ctr, long long n, cudaStream_t s);
cudaError_t launch_upload(const BoxDev& b, const double* pos, const double* vel,
                          const int* type, int set_vel, Launch l);
cudaError_t launch_download(const BoxDev& b, double* pos, double* vel, int* img, Launch l);
cudaError_t launch_force_out(const BoxDev& b, double* f, Launch l);
cudaError_t launch_materialize(const BoxDev& b, Launch l);
cudaError_t launch_get_nlist(const BoxDev& b, int* count, long long* nbr, long long cap,
                             double* pos, Launch l);
