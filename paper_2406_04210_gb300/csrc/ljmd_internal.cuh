// ljmd_internal.cuh -- device data layout and kernel launchers of libljmd.
//
// Layout in HBM (one batch of nrep replicas, np particle slots):
//   * particles of replica r occupy slots [p_off, p_off + n) with p_off a
//     multiple of 32; slots are sorted by (cell, user index) at every list
//     build (particle binning, Sec. 3 "Code structure").
//   * the integrator state of a particle is its cell id plus the offset from
//     that cell's centre ("cell-relative offset"), so FP32 copies of the
//     offsets keep ~1e-7 absolute resolution whatever the box size.  In
//     MD_PREC_MIXED_DS the offsets and velocities are double-single pairs
//     (hi, lo) of FP32; otherwise FP64.
//   * posq[p] = (float offset x, y, z, type bits) feeds the FP32 pair kernels.
//   * Verlet lists (Sec. 3) are 32-bit entries (stencil code << 27 | j) in a
//     warp-blocked layout: entry s of particle p lives at
//     nbr[(p >> 5) * K * 32 + s * 32 + (p & 31)], so the 32 lists of a warp
//     are one contiguous K*128-byte block and each slot load is coalesced.
//     The stencil code k = 9(dz+1) + 3(dy+1) + (dx+1) names the image shift
//     of j's cell relative to i's cell, so d_ij = (o_i - o_j) - k_shift.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define LJ_MAXT 8
#define LJ_IDX_BITS 27
#define LJ_IDX_MASK ((1u << LJ_IDX_BITS) - 1u)
#define LJ_CHUNK 128           // particles per work item (one CTA pass)

// error word bits (err[0]); err[1] = largest list length seen
#define LJ_ERRBIT_CAPACITY 1
#define LJ_ERRBIT_NONFINITE 2
#define LJ_ERRBIT_TIMEOUT 4

// integrate kernel modes
#define LJ_STEP_FIRST 0        // half kick + drift
#define LJ_STEP_MID 1          // finalize previous step + half kick + drift
#define LJ_STEP_LAST 2         // finalize

struct RepDev {
    double L[3];
    double ell[3];             // cell edge lengths
    double inv_ell[3];
    float ellf[3];
    int nc[3];
    int cell_off, ncell;
    int p_off, n;              // first slot, real particles
    int u_off;                 // first user index
    int chunk_off, nchunk;     // work items of this replica
    int pad;
};

// pair parameters, FP32 and FP64 copies: per type pair (a*nt+b)
struct LJDev {
    int nt;
    int shift_on;
    float sig2[LJ_MAXT * LJ_MAXT], eps48[LJ_MAXT * LJ_MAXT], eps4[LJ_MAXT * LJ_MAXT];
    float rc2[LJ_MAXT * LJ_MAXT], shift[LJ_MAXT * LJ_MAXT];
    double dsig2[LJ_MAXT * LJ_MAXT], deps48[LJ_MAXT * LJ_MAXT], deps4[LJ_MAXT * LJ_MAXT];
    double drc2[LJ_MAXT * LJ_MAXT], dshift[LJ_MAXT * LJ_MAXT];
    double deps[LJ_MAXT * LJ_MAXT], dsig[LJ_MAXT * LJ_MAXT];
};

// Everything a kernel needs, passed by value.
struct BoxDev {
    int nrep, np, nchunk, ncell;
    int K;                     // list capacity (slots per particle)
    int prec;                  // md_precision
    int nt;                    // species count
    float disp_thr2;           // rebuild when |displacement|^2 > this (FP32)
    float band;                // FP64 recheck band on |d|^2 around rl^2
    float rl2f;
    double rl2;
    const RepDev* rep;
    const int4* chunk;         // (rep, p_begin, p_end, chunk index)
    const LJDev* lj;
    // particle arrays (sorted order)
    float4* posq;
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
    double* velB;
    int* imgB;
    int* uidB;
    int* typeB;
    int* cellB;
    int* perm;                 // slot -> old index, during a rebuild
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
    unsigned long long* nbuild;
    int* err;
    // per-chunk FP64 partial sums
    double* part_f;            // [chunk*2 + 0] = E_pot share, [+1] = W share
    double* part_k;            // [chunk] = E_kin share
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

__device__ __forceinline__ bool rep_needs_rebuild(const BoxDev& b, int r)
{
    return b.rebuild_req[r] != 0 || __uint_as_float(b.disp_max[r]) > b.disp_thr2;
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
cudaError_t launch_sortgather(const BoxDev& b, Launch l);
cudaError_t launch_nlist(const BoxDev& b, Launch l);

// k_force.cu
cudaError_t launch_force(const BoxDev& b, int energy, Launch l);
cudaError_t launch_thermo(const BoxDev& b, double* out, int with_kin, Launch l);
cudaError_t launch_hvp(const BoxDev& b, const double* u, double* hu, double* part_g, Launch l);

// k_integrate.cu
cudaError_t launch_integrate(const BoxDev& b, int mode, int energy, double dt, Launch l);
cudaError_t launch_upload(const BoxDev& b, const double* pos, const double* vel,
                          const int* type, int set_vel, Launch l);
cudaError_t launch_download(const BoxDev& b, double* pos, double* vel, int* img, Launch l);
cudaError_t launch_force_out(const BoxDev& b, double* f, Launch l);
cudaError_t launch_materialize(const BoxDev& b, Launch l);
cudaError_t launch_get_nlist(const BoxDev& b, int* count, long long* nbr, long long cap,
                             double* pos, Launch l);
