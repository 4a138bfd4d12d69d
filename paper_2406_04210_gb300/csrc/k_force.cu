// k_force.cu -- truncated Lennard-Jones pair force, energy and virial over the
// Verlet list (Sec. 4: Lennard-Jones pair forces; Sec. 5, Truncated Force
// Performance Study: the force kernel over Verlet lists is ~60 % of the run
// time and is memory-latency sensitive -- the CUDA version there reads packed
// float4 particle data through the texture path).
//
// The threads of particle i, in cell-sorted order, walk its list:
//   d_ij = (o_i - o_j) - shift(k)       cell-relative offsets, FP32
//   F_i += 48 eps/r^2 [(s/r)^12 - (s/r)^6/2] d_ij      for r^2 < rc^2
// E_pot and W are summed per thread in the kernel's real type, reduced per
// warp (list kernels) or per work item (all pairs) in FP64 (each pair is
// seen twice in a full list: factor 1/2).
#include "ljmd_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum two doubles over the block; valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& c, double (*s)[32])
{
    a = warp_sum_d(a);
    c = warp_sum_d(c);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][warp] = a;
        s[1][warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += s[0][k];
            c += s[1][k];
        }
    }
    __syncthreads();
}

// One pair term of the FP32 force: accumulates f d into (fx, fy, fz) and,
// with ENERGY, the pair energy and virial; the term is masked (not branched)
// by the cutoff test, so the threads of a particle never diverge.  Entries
// past a row's count name the sentinel slot, whose distance fails the test.
template <bool MONO, bool ENERGY>
__device__ __forceinline__ void pair_f32(unsigned ent, const float4& pj, const float4& pi, int ti,
                                         const float3& ell, const float4* s_lj, const float* s_rc2,
                                         const float* s_esh, int nt, const float4& mlj, float mrc2,
                                         float mesh, float& fx, float& fy, float& fz, float& e, float& vir)
{
    // d = (o_i - o_j) - (dx, dy, dz) * ell, one rounding per component; the
    // x and y parts as FP32 pairs (a gathered float4 holds them as a register
    // pair), computed negated: -d = (o_j - o_i) + (dx, dy) * ell, exactly
    // the negation of the scalar form
    const float2 uxy = __fadd2_rn(make_float2(__uint_as_float(0x4B400000u | ((ent >> 26) & 3u)),
                                              __uint_as_float(0x4B400000u | ((ent >> 28) & 3u))),
                                  make_float2(-12582913.0f, -12582913.0f));
    const float2 tq = __fadd2_rn(make_float2(pj.x, pj.y), make_float2(-pi.x, -pi.y));
    const float2 dq = __ffma2_rn(uxy, make_float2(ell.x, ell.y), tq);
    const float dz = fmaf(-entry_unit(ent, 30), ell.z, pi.z - pj.z);
    const float2 sq = __fmul2_rn(dq, dq);
    const float r2 = fmaf(dz, dz, sq.x + sq.y);
    float4 c;
    float rc2, esh;
    if (MONO) {
        c = mlj;
        rc2 = mrc2;
        esh = mesh;
    } else {
        const int pp = ti * nt + __float_as_int(pj.w);
        c = s_lj[pp];
        rc2 = s_rc2[pp];
        esh = ENERGY ? s_esh[pp] : 0.f;
    }
    const float r2i = rcp_approx(r2);
    const float r6i = r2i * r2i * r2i;
    // c = (48 eps sigma^12, 24 eps sigma^6, 4 eps sigma^12, 4 eps sigma^6)
    float f = r2i * r6i * fmaf(c.x, r6i, -c.y);
    const bool in = r2 < rc2;
    f = in ? f : 0.f;
    fx = fmaf(-f, dq.x, fx);
    fy = fmaf(-f, dq.y, fy);
    fz = fmaf(f, dz, fz);
    if (ENERGY) {
        const float u = fmaf(r6i, fmaf(c.z, r6i, -c.w), -esh);
        e += in ? u : 0.f;
        vir = fmaf(f, r2, vir);
    }
}

// FP32 pair force (Sec. 4/5), one 128-particle chunk per block pass, LJ_TPP
// (4) threads per particle.  A particle's row is read in blocks of
// LJ_ROW_BLOCK (16) entries, the last block's entries past the count
// replaced by the sentinel slot; thread l8 of the particle takes entries
// 4 l8 .. 4 l8 + 3 of each block with one 16-byte load (the next block's
// load in flight while this one is computed), gathers the four neighbours'
// FP32 offsets through L1 (four gathers in flight, two independent pair
// chains) and the four threads combine their partial forces with shuffles.
// The kernel is bound by gather latency: resident warps matter more than
// gathers in flight per thread.  Six blocks of 256 per SM (40 registers, no
// spills) measured 11 % faster than four (64 registers), and eight gathers
// in flight at three blocks 9 % slower.  On the 4M-particle fluid 4 threads
// per particle x 4 entries per thread measured fastest among 2/4/8 x 2/4/8.
// MONO: a single species, its pair constants read from the kernel
// parameters.  SINGLE (MONO and one replica): the cell edge from the
// parameters too and one pair chain, 32 registers, eight blocks per SM.
static_assert(LJ_TPP * 4 == LJ_ROW_BLOCK, "a row block is one 16-byte load per thread of a particle");
template <bool MONO, bool ENERGY, bool SINGLE>
__global__ void __launch_bounds__(LJ_FORCE_THREADS, SINGLE ? 8 : 6) k_force_f32(BoxDev b)
{
    __shared__ float4 s_lj[LJ_MAXT * LJ_MAXT];   // c12, c6, e12, e6
    __shared__ float s_rc2[LJ_MAXT * LJ_MAXT];
    __shared__ float s_esh[LJ_MAXT * LJ_MAXT];
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
        s_lj[k] = make_float4(lj->c12[k], lj->c6[k], lj->e12[k], lj->e6[k]);
        s_rc2[k] = lj->rc2[k];
        s_esh[k] = lj->shift[k];
    }
    __syncthreads();   // the pair tables are complete (the block's only barrier)
    const float4 mlj = b.c1;
    const float mrc2 = b.rc2_1;
    const float mesh = b.esh_1;
    const int K = b.K;
    const int grp = threadIdx.x / LJ_TPP, l8 = threadIdx.x % LJ_TPP;
    const float4* __restrict__ posq = b.posq;
    const unsigned sent = entry_make(13, b.np);
    int cur_r = -1;
    float3 ell = make_float3(0.f, 0.f, 0.f);
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        const int4 ch = b.chunk[w];
        const int r = ch.x;
        if (SINGLE) {
            ell = b.ell1;
        } else if (r != cur_r) {                // block-uniform
            const RepDev& R = b.rep[r];
            ell = make_float3(R.ellf[0], R.ellf[1], R.ellf[2]);
            cur_r = r;
        }
        if (threadIdx.x == 0) {
            if (w == 0) *b.any_req = 0;         // the list update of this step has run
            if (w == b.rep[r].chunk_off) {      // clear the replica's rebuild triggers
                b.disp_max[r] = 0u;
                b.rebuild_req[r] = 0;
            }
        }
        float e = 0.f, vir = 0.f;
        for (int base = ch.y; base < ch.z; base += LJ_FORCE_THREADS / LJ_TPP) {
            const int p = base + grp;
            const bool act = p < ch.z;
            float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
            int cnt = 0;
            const uint4* L = reinterpret_cast<const uint4*>(b.nbr + (size_t)K * p) + l8;
            uint4 cur = make_uint4(0u, 0u, 0u, 0u);
            if (act) {
                pi = posq[p];
                cnt = min(b.nbr_count[p], K);
                cur = __ldcs(L);   // the row's first block (K >= 16 slots), in flight with the count
            }
            const int nblk = (cnt + LJ_ROW_BLOCK - 1) / LJ_ROW_BLOCK;
            const int ti = __float_as_int(pi.w);
            float fx = 0.f, fy = 0.f, fz = 0.f, fx2 = 0.f, fy2 = 0.f, fz2 = 0.f;
            // the second pair chain: independent partial forces, or (SINGLE,
            // registers for occupancy) the first chain itself
            float& gx = SINGLE ? fx : fx2;
            float& gy = SINGLE ? fy : fy2;
            float& gz = SINGLE ? fz : fz2;
            // four entries: four gathers in flight
            auto block4 = [&](const uint4& q) {
                const float4 p0 = __ldg(posq + (q.x & LJ_IDX_MASK));
                const float4 p1 = __ldg(posq + (q.y & LJ_IDX_MASK));
                const float4 p2 = __ldg(posq + (q.z & LJ_IDX_MASK));
                const float4 p3 = __ldg(posq + (q.w & LJ_IDX_MASK));
                pair_f32<MONO, ENERGY>(q.x, p0, pi, ti, ell, s_lj, s_rc2, s_esh, nt, mlj, mrc2, mesh,
                                       fx, fy, fz, e, vir);
                pair_f32<MONO, ENERGY>(q.y, p1, pi, ti, ell, s_lj, s_rc2, s_esh, nt, mlj, mrc2, mesh,
                                       gx, gy, gz, e, vir);
                pair_f32<MONO, ENERGY>(q.z, p2, pi, ti, ell, s_lj, s_rc2, s_esh, nt, mlj, mrc2, mesh,
                                       fx, fy, fz, e, vir);
                pair_f32<MONO, ENERGY>(q.w, p3, pi, ti, ell, s_lj, s_rc2, s_esh, nt, mlj, mrc2, mesh,
                                       gx, gy, gz, e, vir);
            };
            if (nblk > 0) {
                for (int blk = 1; blk < nblk; ++blk) {
                    const uint4 nxt = __ldcs(L + blk * LJ_TPP);   // in flight during this block
                    block4(cur);
                    cur = nxt;
                }
                // the row's last block: entries past the count (stale or
                // never written) name the sentinel slot
                const int lim = cnt - ((nblk - 1) * LJ_ROW_BLOCK + 4 * l8);
                cur.x = lim > 0 ? cur.x : sent;
                cur.y = lim > 1 ? cur.y : sent;
                cur.z = lim > 2 ? cur.z : sent;
                cur.w = lim > 3 ? cur.w : sent;
                block4(cur);
            }
            if (!SINGLE) {
                fx += fx2;
                fy += fy2;
                fz += fz2;
            }
#pragma unroll
            for (int o = LJ_TPP / 2; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
            }
            if (act && l8 == 0) {
                b.force4[p] = make_float4(fx, fy, fz, 0.f);
                if (!isfinite(fx + fy + fz)) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
            }
        }
        if (ENERGY) {
            // one (E_pot, W) share per warp and chunk, no block barrier: the
            // warps of a block run ahead into the next chunk independently.
            // The warp sum is double-single (two FP32 words per partial
            // sum): FP64-class precision on the FP32 pipe, since FP64 adds
            // are scarce on this GPU.  The share is stored as the (hi, lo)
            // pair itself (pf_ds), halved exactly; the reduction converts
            const float2 de = warp_sum_ds2(e), dw = warp_sum_ds2(vir);
            if ((threadIdx.x & 31) == 0) {
                const size_t q = (size_t)w * LJ_FORCE_WARPS + (threadIdx.x >> 5);
                reinterpret_cast<float4*>(b.part_f)[q] =
                    make_float4(0.5f * de.x, 0.5f * de.y, 0.5f * dw.x, 0.5f * dw.y);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled FP32 pair force (Sec. 4/5: the same forces, energy and virial as
// k_force_f32; Sec. 5 finds the force kernel bound by fetching neighbour
// data, which here comes from shared memory).  The work items are bricks
// of up to 2 x 2 x 2 cells.  A producer warp stages the FP32 offsets of a
// brick's neighbourhood (its cells and the layer of cells around them, up to
// 64 cells) as x, y and z planes of a shared-memory tile, each moved into
// the frame of the brick's centre by one FMA (q_j = o_j + a ell, a a
// multiple of 1/2, one rounding), double-buffered; the consumer warps walk
// the brick's particles' list rows, LJ_TPP threads per particle, four
// entries per thread and 16-entry row block.  An entry (stencil digits of neighbour cell k, slot j) names the
// tile element j - start + base of the tile cell at the particle's cell plus
// k: its byte address is (entry << 2) plus a table word of the particle's
// cell indexed by the digits, which also cancels what the shift leaves of
// the digits -- one shift-add per entry, no decode and no image shift per
// pair.  Pairs are evaluated two at a time with FP32-pair arithmetic on
// d' = q_j - p_i = -d_ij (p_i = o_i + a_i ell, the sums negated at the
// end).  Brick edges are 2 cells only where a tile coordinate stays below 8
// (one rounding of 2^-22 at most); a brick whose neighbourhood holds more
// than LJ_BRICK_TILE particles is evaluated from global memory as in
// k_force_f32.  Energy and virial: one double-single (E_pot, W) share per
// warp and brick, summed in FP64 by k_thermo in a fixed order.
// ---------------------------------------------------------------------------

// x, y, z of the tile element at byte address a (planes PL bytes apart)
template <int PL>
__device__ __forceinline__ void tile_xyz(uint32_t a, float& x, float& y, float& z)
{
    asm("ld.shared.f32 %0, [%3];\n\t"
        "ld.shared.f32 %1, [%3+%4];\n\t"
        "ld.shared.f32 %2, [%3+%5];"
        : "=f"(x), "=f"(y), "=f"(z)
        : "r"(a), "n"(PL), "n"(2 * PL));
}
template <int PL>
__device__ __forceinline__ int tile_type(uint32_t a)
{
    int t;
    asm("ld.shared.b32 %0, [%1+%2];" : "=r"(t) : "r"(a), "n"(3 * PL));
    return t;
}

struct PairAcc2 {
    float2 fx, fy, fz, e, w;
};

// Two pair terms (tile elements at a0, a1) against particle i (n = -p_i),
// accumulated as FP32 pairs; masked, not branched, by the cutoff test.
template <bool MONO, bool ENERGY, int PL>
__device__ __forceinline__ void tile_pair2(uint32_t a0, uint32_t a1, const float2& nx, const float2& ny,
                                           const float2& nz, int ti, int nt, const float4* s_lj,
                                           const float* s_rc2, const float* s_esh, const float4& mlj,
                                           float mrc2, float mesh, PairAcc2& A)
{
    float x0, y0, z0, x1, y1, z1;
    tile_xyz<PL>(a0, x0, y0, z0);
    tile_xyz<PL>(a1, x1, y1, z1);
    const float2 dx = __fadd2_rn(make_float2(x0, x1), nx);
    const float2 dy = __fadd2_rn(make_float2(y0, y1), ny);
    const float2 dz = __fadd2_rn(make_float2(z0, z1), nz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    float2 c12, nc6, e12, ne6, rc2, nesh;
    if (MONO) {
        c12 = make_float2(mlj.x, mlj.x);
        nc6 = make_float2(-mlj.y, -mlj.y);
        e12 = make_float2(mlj.z, mlj.z);
        ne6 = make_float2(-mlj.w, -mlj.w);
        rc2 = make_float2(mrc2, mrc2);
        nesh = make_float2(-mesh, -mesh);
    } else {
        const int p0 = ti * nt + tile_type<PL>(a0), p1 = ti * nt + tile_type<PL>(a1);
        const float4 q0 = s_lj[p0], q1 = s_lj[p1];
        c12 = make_float2(q0.x, q1.x);
        nc6 = make_float2(-q0.y, -q1.y);
        e12 = make_float2(q0.z, q1.z);
        ne6 = make_float2(-q0.w, -q1.w);
        rc2 = make_float2(s_rc2[p0], s_rc2[p1]);
        nesh = ENERGY ? make_float2(-s_esh[p0], -s_esh[p1]) : make_float2(0.f, 0.f);
    }
    const float2 ri = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    const float2 r6 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
    float2 f = __fmul2_rn(__fmul2_rn(ri, r6), __ffma2_rn(c12, r6, nc6));
    const bool in0 = r2.x < rc2.x, in1 = r2.y < rc2.y;
    f.x = in0 ? f.x : 0.f;
    f.y = in1 ? f.y : 0.f;
    A.fx = __ffma2_rn(f, dx, A.fx);
    A.fy = __ffma2_rn(f, dy, A.fy);
    A.fz = __ffma2_rn(f, dz, A.fz);
    if (ENERGY) {
        float2 u = __ffma2_rn(r6, __ffma2_rn(e12, r6, ne6), nesh);
        u.x = in0 ? u.x : 0.f;
        u.y = in1 ? u.y : 0.f;
        A.e = __fadd2_rn(A.e, u);
        A.w = __ffma2_rn(f, r2, A.w);
    }
}

// tile address of entry e for the particle's address table D
__device__ __forceinline__ uint32_t tile_addr(uint32_t e, const uint32_t* D) { return (e << 2) + D[e >> 26]; }

static_assert(LJ_BRICK_WARPS == LJ_FORCE_WARPS, "per-brick shares in the chunk kernel's share stride");
constexpr int kBrickThreads = LJ_BRICK_THREADS;          // consumer threads
constexpr int kBrickWarps = kBrickThreads / 32;          // consumer warps (the producer is warp kBrickWarps)
constexpr int kBrickPass = kBrickThreads / LJ_TPP;       // particles per consumer pass

__device__ __forceinline__ void mbar_arrive1(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Dynamic shared memory of k_force_tile_f32: two buffers of NPL planes.
constexpr size_t tile_buf_bytes(bool mono) { return (size_t)(mono ? 3 : 4) * (LJ_BRICK_TILE + 1) * 4; }

// Producer warp kBrickWarps stages brick k + 1 (tile planes, brick-cell
// tables, address tables) into one buffer while the consumer warps compute
// brick k from the other; full[buf] (32 arrivals, the producer's lanes) and
// empty[buf] (kBrickThreads arrivals, the consumers) hand the buffers over.
// Every wait is bounded: on a timeout the warp records LJ_ERRBIT_TIMEOUT and
// leaves, and the others then time out in turn.
template <bool MONO, bool ENERGY>
__global__ void __launch_bounds__(LJ_BRICK_THREADS + 32, 4) k_force_tile_f32(BoxDev b)
{
    constexpr int T = LJ_BRICK_TILE;
    constexpr int NPL = MONO ? 3 : 4;   // x, y, z (and type) planes
    constexpr int PL = (T + 1) * 4;     // bytes per plane; element T of each is the sentinel
    constexpr int BUF = NPL * PL;       // bytes per buffer
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float s_dyn[];   // [2][NPL][T + 1]
    __shared__ uint32_t s_D[2][8][64];  // per buffer, brick cell and stencil-digit code: tile address term
    __shared__ int s_pc[2][9], s_cs[2][8], s_nb[2], s_tiled[2];   // per buffer: brick cells, particles
    __shared__ int s_tb[64], s_ts[64], s_tn[64];                  // producer: tile cells
    __shared__ unsigned long long s_full[2], s_empty[2];
    __shared__ float4 s_lj[MONO ? 1 : LJ_MAXT * LJ_MAXT];
    __shared__ float s_rc2[MONO ? 1 : LJ_MAXT * LJ_MAXT];
    __shared__ float s_esh[MONO ? 1 : LJ_MAXT * LJ_MAXT];
    const int nt = b.nt;
    if (!MONO) {
        const LJDev* lj = b.lj;
        for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
            s_lj[k] = make_float4(lj->c12[k], lj->c6[k], lj->e12[k], lj->e6[k]);
            s_rc2[k] = lj->rc2[k];
            s_esh[k] = lj->shift[k];
        }
    }
    if (threadIdx.x < 2 * NPL) {   // sentinels: far offsets, type 0
        const int q = threadIdx.x % NPL;
        s_dyn[(threadIdx.x / NPL) * NPL * (T + 1) + q * (T + 1) + T] = q < 3 ? LJ_SENTINEL_OFF : 0.f;
    }
    if (threadIdx.x == 0) {
        mbar_init(&s_full[0], 32);
        mbar_init(&s_full[1], 32);
        mbar_init(&s_empty[0], kBrickThreads);
        mbar_init(&s_empty[1], kBrickThreads);
    }
    __syncthreads();   // the block's only barrier: the roles part here
    const uint32_t X0 = (uint32_t)__cvta_generic_to_shared(s_dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float4* __restrict__ posq = b.posq;

    if (warp == kBrickWarps) {
        // ---------------- producer ----------------
        int k = 0;
        for (int bi = blockIdx.x; bi < b.nbrick; bi += gridDim.x, ++k) {
            const int buf = k & 1;
            if (k >= 2 && !mbar_wait(&s_empty[buf], ((k >> 1) - 1) & 1)) {
                if (lane == 0) atomicOr(&b.err[0], LJ_ERRBIT_TIMEOUT);
                return;
            }
            const int4 B = b.brick[bi];
            const int r = B.x;
            const RepDev& R = b.rep[r];
            if (lane == 0) {
                if (bi == 0) *b.any_req = 0;   // the list update of this step has run
                if (B.y == 0 && B.z == 0 && B.w == 0) {   // the replica's first brick: clear its rebuild triggers
                    b.disp_max[r] = 0u;
                    b.rebuild_req[r] = 0;
                }
            }
            const int ex = min(R.br[0], R.nc[0] - B.y), ey = min(R.br[1], R.nc[1] - B.z),
                      ez = min(R.br[2], R.nc[2] - B.w);
            const int tx = ex + 2, txy = tx * (ey + 2), ntc = txy * (ez + 2), nbc = ex * ey * ez;
            const int sx = ex - 1, sy = ey - 1;   // brick cell cl = u + ex (v + ey w): u = cl & sx, ...
            const float3 ell = make_float3(R.ellf[0], R.ellf[1], R.ellf[2]);
            // tile coordinate t along an axis (brick cell u is t = u + 1): its
            // offset in cells from the brick centre, t - (extent + 1) / 2
            const float hx = 0.5f * (float)(ex + 1), hy = 0.5f * (float)(ey + 1), hz = 0.5f * (float)(ez + 1);
            // tile cells 2 lane and 2 lane + 1: first slot and particles, then
            // their bases (exclusive prefix over the tile)
            int js[2] = {0, 0}, nk[2] = {0, 0};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = 2 * lane + u;
                if (t < ntc) {
                    const int a = t % tx, c = t / txy, bb = (t / tx) - c * (ey + 2);
                    const int cn = R.cell_off + wrapi(B.y - 1 + a, R.nc[0]) +
                                   R.nc[0] * (wrapi(B.z - 1 + bb, R.nc[1]) + R.nc[1] * wrapi(B.w - 1 + c, R.nc[2]));
                    js[u] = b.cell_start[cn];
                    nk[u] = b.cell_end[cn] - js[u];
                }
            }
            int incl = nk[0] + nk[1];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const int e0 = incl - nk[0] - nk[1];
            s_tb[2 * lane] = e0;
            s_tb[2 * lane + 1] = e0 + nk[0];
            s_ts[2 * lane] = js[0];
            s_ts[2 * lane + 1] = js[1];
            s_tn[2 * lane] = nk[0];
            s_tn[2 * lane + 1] = nk[1];
            const bool tiled = __shfl_sync(FULL, incl, 31) <= T;
            __syncwarp();
            // brick cells (lane < 8): first slot and particle prefix
            int n8 = 0;
            if (lane < nbc) {
                const int u = lane & sx, v = (lane >> sx) & sy, w = lane >> (sx + sy);
                const int t = (u + 1) + tx * (v + 1) + txy * (w + 1);
                s_cs[buf][lane] = s_ts[t];
                n8 = s_tn[t];
            }
            int inc8 = n8;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int t = __shfl_up_sync(FULL, inc8, o);
                if (lane >= o) inc8 += t;
            }
            if (lane < 8) s_pc[buf][lane + 1] = inc8;   // lanes past the brick's cells add nothing
            const int npb = __shfl_sync(FULL, inc8, 7);
            if (lane == 0) {
                s_pc[buf][0] = 0;
                s_nb[buf] = npb;
                s_tiled[buf] = tiled ? 1 : 0;
            }
            if (tiled) {
                float* const P = s_dyn + buf * NPL * (T + 1);
                const uint32_t Xb = X0 + (uint32_t)(buf * BUF);
                // rows of the tile (tile cells along x at one y, z), 4 elements
                // per lane in flight
                const int nrow = (ey + 2) * (ez + 2);
                for (int rr = 0; rr < nrow; ++rr) {
                    const int t0 = rr * tx;
                    const int rb = s_tb[t0], re = s_tb[t0 + tx - 1] + s_tn[t0 + tx - 1];
                    const float ay = (float)(rr % (ey + 2)) - hy, az = (float)(rr / (ey + 2)) - hz;   // exact
                    for (int f0 = rb; f0 < re; f0 += 128) {
                        float4 v[4];
                        int at[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e = f0 + 32 * u + lane;
                            int a = 0;   // the tile cell of element e along the row
#pragma unroll
                            for (int c = 1; c < 4; ++c) a += (c < tx && s_tb[t0 + c] <= e) ? 1 : 0;
                            at[u] = a;
                            v[u] = e < re ? posq[s_ts[t0 + a] + (e - s_tb[t0 + a])] : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e = f0 + 32 * u + lane;
                            if (e < re) {
                                P[e] = fmaf((float)at[u] - hx, ell.x, v[u].x);
                                P[(T + 1) + e] = fmaf(ay, ell.y, v[u].y);
                                P[2 * (T + 1) + e] = fmaf(az, ell.z, v[u].z);
                                if (!MONO) P[(NPL - 1) * (T + 1) + e] = v[u].w;   // type bits
                            }
                        }
                    }
                }
                // address tables: brick cell cl, stencil cell k
                for (int t = lane; t < nbc * 27; t += 32) {
                    const int cl = t / 27, kk = t - 27 * cl;
                    const int u = cl & sx, v = (cl >> sx) & sy, w = cl >> (sx + sy);
                    const uint32_t dxd = kk % 3, dyd = (kk / 3) % 3, dzd = kk / 9;
                    const int tc = (u + (int)dxd) + tx * (v + (int)dyd) + txy * (w + (int)dzd);
                    // (entry << 2) = 4 j + (dx digit << 28) + (dy digit << 30) mod 2^32
                    s_D[buf][cl][(dzd << 4) | (dyd << 2) | dxd] =
                        Xb + 4u * (uint32_t)(s_tb[tc] - s_ts[tc]) - (dxd << 28) - (dyd << 30);
                }
            }
            mbar_arrive1(&s_full[buf]);   // every producer lane: its stores precede the arrival
        }
        return;
    }

    // ---------------- consumers ----------------
    const int grp = threadIdx.x / LJ_TPP, l4 = threadIdx.x % LJ_TPP;
    const int K = b.K;
    const float4 mlj = b.c1;
    const float mrc2 = b.rc2_1, mesh = b.esh_1;
    const unsigned sent_ent = entry_make(13, b.np);
    int k = 0;
    for (int bi = blockIdx.x; bi < b.nbrick; bi += gridDim.x, ++k) {
        const int buf = k & 1;
        if (!mbar_wait(&s_full[buf], (k >> 1) & 1)) {
            if (lane == 0) atomicOr(&b.err[0], LJ_ERRBIT_TIMEOUT);
            return;
        }
        const int4 B = b.brick[bi];
        const RepDev& R = b.rep[B.x];
        const int ex = min(R.br[0], R.nc[0] - B.y), ey = min(R.br[1], R.nc[1] - B.z),
                  ez = min(R.br[2], R.nc[2] - B.w);
        const int nbc = ex * ey * ez, sx = ex - 1, sy = ey - 1;
        const float3 ell = make_float3(R.ellf[0], R.ellf[1], R.ellf[2]);
        const float hx = 0.5f * (float)(ex + 1), hy = 0.5f * (float)(ey + 1), hz = 0.5f * (float)(ez + 1);
        const bool tiled = s_tiled[buf] != 0;
        const int npb = s_nb[buf];
        const uint32_t SENT = X0 + (uint32_t)(buf * BUF) + 4u * (uint32_t)T;
        float e_acc = 0.f, w_acc = 0.f;   // this thread's energy and virial over the brick
        for (int ib = 0; ib < npb; ib += kBrickPass) {
            if (ib + (32 / LJ_TPP) * warp >= npb) break;   // warp-uniform: none of its particles here or later
            const int slot = ib + grp;
            const bool act = slot < npb;
            // its brick cell: the last cl < nbc with s_pc[cl] <= slot (prefix non-decreasing)
            const int* pc = s_pc[buf];
            int cl = (4 < nbc && pc[4] <= slot) ? 4 : 0;
            cl += (cl + 2 < nbc && pc[cl + 2] <= slot) ? 2 : 0;
            cl += (cl + 1 < nbc && pc[cl + 1] <= slot) ? 1 : 0;
            const int p = act ? s_cs[buf][cl] + (slot - pc[cl]) : 0;   // no load for an idle group
            const float4 pi = act ? posq[p] : make_float4(0.f, 0.f, 0.f, 0.f);
            const uint4* L = reinterpret_cast<const uint4*>(b.nbr + (size_t)K * p) + l4;
            const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
            // the row's first two blocks (inside the row's K >= 16 slots), in
            // flight with the count; later blocks two ahead
            uint4 cur = act ? __ldcs(L) : z4;
            uint4 nx1 = act && K > LJ_ROW_BLOCK ? __ldcs(L + LJ_TPP) : z4;
            const int cnt = act ? min(b.nbr_count[p], K) : 0;
            const int nblk = (cnt + LJ_ROW_BLOCK - 1) / LJ_ROW_BLOCK;
            const int ti = __float_as_int(pi.w);
            const int lim = cnt - ((nblk - 1) * LJ_ROW_BLOCK + 4 * l4);   // valid entries of the last block
            PairAcc2 A;
            A.fx = A.fy = A.fz = A.e = A.w = make_float2(0.f, 0.f);
            if (tiled) {
                const int u = cl & sx, v = (cl >> sx) & sy, w = cl >> (sx + sy);
                // p_i in the brick frame: one rounding
                const float px = fmaf((float)(u + 1) - hx, ell.x, pi.x), py = fmaf((float)(v + 1) - hy, ell.y, pi.y),
                            pz = fmaf((float)(w + 1) - hz, ell.z, pi.z);
                const float2 nx = make_float2(-px, -px), ny = make_float2(-py, -py), nz = make_float2(-pz, -pz);
                const uint32_t* D = s_D[buf][cl];
                for (int blk = 0; blk + 1 < nblk; ++blk) {
                    const uint4 nx2 = blk + 2 < nblk ? __ldcs(L + (blk + 2) * LJ_TPP) : z4;   // two ahead
                    tile_pair2<MONO, ENERGY, PL>(tile_addr(cur.x, D), tile_addr(cur.y, D), nx, ny, nz, ti, nt, s_lj,
                                                 s_rc2, s_esh, mlj, mrc2, mesh, A);
                    tile_pair2<MONO, ENERGY, PL>(tile_addr(cur.z, D), tile_addr(cur.w, D), nx, ny, nz, ti, nt, s_lj,
                                                 s_rc2, s_esh, mlj, mrc2, mesh, A);
                    cur = nx1;
                    nx1 = nx2;
                }
                if (nblk > 0) {   // the last block: entries past the count name the sentinel
                    const uint32_t a0 = lim > 0 ? tile_addr(cur.x, D) : SENT;
                    const uint32_t a1 = lim > 1 ? tile_addr(cur.y, D) : SENT;
                    const uint32_t a2 = lim > 2 ? tile_addr(cur.z, D) : SENT;
                    const uint32_t a3 = lim > 3 ? tile_addr(cur.w, D) : SENT;
                    tile_pair2<MONO, ENERGY, PL>(a0, a1, nx, ny, nz, ti, nt, s_lj, s_rc2, s_esh, mlj, mrc2, mesh, A);
                    tile_pair2<MONO, ENERGY, PL>(a2, a3, nx, ny, nz, ti, nt, s_lj, s_rc2, s_esh, mlj, mrc2, mesh, A);
                }
            } else {   // neighbourhood larger than the tile: gathers from global memory
                float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, vir = 0.f;
                for (int blk = 0; blk < nblk; ++blk) {
                    const bool last = blk + 1 == nblk;
                    const uint4 nx2 = blk + 2 < nblk ? __ldcs(L + (blk + 2) * LJ_TPP) : z4;
                    uint32_t q[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const unsigned ek = (!last || lim > kk) ? q[kk] : sent_ent;
                        const float4 pj = __ldg(posq + (ek & LJ_IDX_MASK));
                        pair_f32<MONO, ENERGY>(ek, pj, pi, ti, ell, s_lj, s_rc2, s_esh, nt, mlj, mrc2, mesh, fx, fy,
                                               fz, e, vir);
                    }
                    cur = nx1;
                    nx1 = nx2;
                }
                // d_ij orientation here: stored negated like the tile path's sums
                A.fx = make_float2(-fx, 0.f);
                A.fy = make_float2(-fy, 0.f);
                A.fz = make_float2(-fz, 0.f);
                A.e = make_float2(e, 0.f);
                A.w = make_float2(vir, 0.f);
            }
            float fx = A.fx.x + A.fx.y, fy = A.fy.x + A.fy.y, fz = A.fz.x + A.fz.y;
            if (ENERGY) {   // idle groups hold zeros
                e_acc += A.e.x + A.e.y;
                w_acc += A.w.x + A.w.y;
            }
#pragma unroll
            for (int o = LJ_TPP / 2; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(FULL, fx, o);
                fy += __shfl_xor_sync(FULL, fy, o);
                fz += __shfl_xor_sync(FULL, fz, o);
            }
            if (act && l4 == 0) {
                b.force4[p] = make_float4(-fx, -fy, -fz, 0.f);
                if (!isfinite(fx + fy + fz)) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
            }
        }
        if (ENERGY) {
            // one (E_pot, W) share per warp and brick, written for every brick
            // (zeros where the warp had no particle): the warp sum in
            // double-single, stored as the (hi, lo) pair, halved exactly
            // (each pair is in two rows of a full list)
            const float2 de = warp_sum_ds2(e_acc), dw = warp_sum_ds2(w_acc);
            if (lane == 0)
                reinterpret_cast<float4*>(b.part_f)[(size_t)bi * kBrickWarps + warp] =
                    make_float4(0.5f * de.x, 0.5f * de.y, 0.5f * dw.x, 0.5f * dw.y);
        }
        mbar_arrive1(&s_empty[buf]);   // every consumer thread: its reads of the buffer precede this
    }
}

// FP64 pair force (MD_PREC_FP64), one thread per particle over 128-particle
// chunks, FP64 cell-relative offsets gathered from global memory.
template <bool ENERGY>
__global__ void __launch_bounds__(LJ_F64_THREADS) k_force_f64(BoxDev b)
{
    __shared__ double s_sh[3][27];
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    const int np = b.np;
    int cur_r = -1;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        const int4 ch = b.chunk[w];
        const int r = ch.x;
        if (r != cur_r) {
            __syncthreads();
            if (threadIdx.x < 27) {
                const RepDev& R = b.rep[r];
                const int k = threadIdx.x;
                s_sh[0][k] = (double)(k % 3 - 1) * R.ell[0];
                s_sh[1][k] = (double)((k / 3) % 3 - 1) * R.ell[1];
                s_sh[2][k] = (double)(k / 9 - 1) * R.ell[2];
            }
            __syncthreads();
            cur_r = r;
        }
        if (threadIdx.x == 0) {
            if (w == 0) *b.any_req = 0;
            if (w == b.rep[r].chunk_off) {
                b.disp_max[r] = 0u;
                b.rebuild_req[r] = 0;
            }
        }
        const int p = ch.y + (int)threadIdx.x;
        double e = 0.0, vir = 0.0;
        if (p < ch.z) {
            double xi = b.off[p], yi = b.off[np + p], zi = b.off[2 * np + p];
            int ti = b.type[p];
            int cnt = min(b.nbr_count[p], b.K);
            const uint32_t* lp = b.nbr + (size_t)b.K * p;
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (int s = 0; s < cnt; ++s) {
                unsigned ent = __ldcs(lp + s);
                int j = (int)(ent & LJ_IDX_MASK);
                int k = entry_k(ent);
                double dx = (xi - __ldg(&b.off[j])) - s_sh[0][k];
                double dy = (yi - __ldg(&b.off[np + j])) - s_sh[1][k];
                double dz = (zi - __ldg(&b.off[2 * np + j])) - s_sh[2][k];
                double r2 = dx * dx + dy * dy + dz * dz;
                int pp = ti * nt + __ldg(&b.type[j]);
                if (r2 < lj->drc2[pp]) {
                    double r2i = 1.0 / r2;
                    double s2 = lj->dsig2[pp] * r2i;
                    double s6 = s2 * s2 * s2;
                    double f = lj->deps48[pp] * r2i * s6 * (s6 - 0.5);
                    fx += f * dx;
                    fy += f * dy;
                    fz += f * dz;
                    if (ENERGY) {
                        e += lj->deps4[pp] * s6 * (s6 - 1.0) - lj->dshift[pp];
                        vir += f * r2;
                    }
                }
            }
            b.force64[p] = fx;
            b.force64[np + p] = fy;
            b.force64[2 * np + p] = fz;
            if (!isfinite(fx + fy + fz)) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
        }
        if (ENERGY) {
            // one (E_pot, W) share per warp and chunk (no block barrier)
            double de = warp_sum_d(0.5 * e), dw = warp_sum_d(0.5 * vir);
            if ((threadIdx.x & 31) == 0) {
                const size_t q = (size_t)w * LJ_F64_WARPS + (threadIdx.x >> 5);
                b.part_f[2 * q] = de;
                b.part_f[2 * q + 1] = dw;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// All pairs (Sec. 4: the untruncated LJ interaction between all particles;
// every cutoff infinite).  Work items are (chunk of 128 particles, slice of
// the replica's particles): a block sums the chunk's forces over its slice
// (LJ_TPP threads per particle, the slice's offsets staged through shared
// memory in tiles) into b.ap_part, and the block that completes a chunk's
// last slice (atomic count) adds the slices in slice order (deterministic).
// With one cell per replica all offsets are from the box centre:
// d = o_i - o_j - L rint((o_i - o_j) / L) is the minimum image.
// ---------------------------------------------------------------------------
constexpr int kAllTile = 1024;
constexpr int kAllThreads = LJ_CHUNK * LJ_TPP;

__device__ __forceinline__ void slice_range(const RepDev& R, int js, int nslice, int& j0, int& j1)
{
    const int len = (R.n + nslice - 1) / nslice;
    j0 = R.p_off + min(R.n, js * len);
    j1 = R.p_off + min(R.n, (js + 1) * len);
}

// The last block of chunk w: true in every thread of it.
__device__ __forceinline__ bool last_slice(const BoxDev& b, int w, int* s_flag)
{
    __syncthreads();   // this block's partials are written
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&b.ap_cnt[w], 1u);
        *s_flag = prev == (unsigned)(b.ap_js - 1);
        if (*s_flag) b.ap_cnt[w] = 0u;
    }
    __syncthreads();
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

template <bool MONO, bool ENERGY>
__global__ void __launch_bounds__(kAllThreads) k_force_all_f32(BoxDev b)
{
    __shared__ float4 s_pos[kAllTile];
    __shared__ float4 s_lj[LJ_MAXT * LJ_MAXT];   // c12, c6, e12, e6
    __shared__ float s_esh[LJ_MAXT * LJ_MAXT];
    __shared__ double s_red[2][32];
    __shared__ int s_flag;
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
        s_lj[k] = make_float4(lj->c12[k], lj->c6[k], lj->e12[k], lj->e6[k]);
        s_esh[k] = lj->shift[k];
    }
    const float4 mlj = make_float4(lj->c12[0], lj->c6[0], lj->e12[0], lj->e6[0]);
    const float mesh = lj->shift[0];
    const int grp = threadIdx.x / LJ_TPP, l4 = threadIdx.x % LJ_TPP;
    const int nitem = b.nchunk * b.ap_js;
    for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int w = it / b.ap_js, js = it % b.ap_js;
        const int4 ch = b.chunk[w];
        const RepDev& R = b.rep[ch.x];
        if (threadIdx.x == 0 && js == 0) {
            if (w == 0) *b.any_req = 0;         // the re-binning of this step has run
            if (w == R.chunk_off) {             // clear the replica's triggers
                b.disp_max[ch.x] = 0u;
                b.rebuild_req[ch.x] = 0;
            }
        }
        const float Lx = (float)R.L[0], Ly = (float)R.L[1], Lz = (float)R.L[2];
        const float ix = (float)(1.0 / R.L[0]), iy = (float)(1.0 / R.L[1]), iz = (float)(1.0 / R.L[2]);
        const int p = ch.y + grp;
        const bool act = p < ch.z;
        const float4 pi = b.posq[act ? p : ch.y];
        const int tb = __float_as_int(pi.w) * nt;
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, vir = 0.f;
        int j0, j1;
        slice_range(R, js, b.ap_js, j0, j1);
        for (int t0 = j0; t0 < j1; t0 += kAllTile) {
            const int nj = min(kAllTile, j1 - t0);
            __syncthreads();   // the previous tile is no longer read
            for (int t = threadIdx.x; t < nj; t += blockDim.x) s_pos[t] = b.posq[t0 + t];
            __syncthreads();
            for (int t = l4; t < nj; t += LJ_TPP) {
                const float4 pj = s_pos[t];
                float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                dx -= Lx * rintf(dx * ix);
                dy -= Ly * rintf(dy * iy);
                dz -= Lz * rintf(dz * iz);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float4 c;
                float esh;
                if (MONO) {
                    c = mlj;
                    esh = mesh;
                } else {
                    const int pp = tb + __float_as_int(pj.w);
                    c = s_lj[pp];
                    esh = ENERGY ? s_esh[pp] : 0.f;
                }
                const float r2i = rcp_approx(r2);
                const float r6i = r2i * r2i * r2i;
                float f = r2i * r6i * fmaf(c.x, r6i, -c.y);
                const bool in = act && t0 + t != p;
                f = in ? f : 0.f;
                fx = fmaf(f, dx, fx);
                fy = fmaf(f, dy, fy);
                fz = fmaf(f, dz, fz);
                if (ENERGY) {
                    const float u = r6i * fmaf(c.z, r6i, -c.w) - esh;
                    e += in ? u : 0.f;
                    vir = fmaf(f, r2, vir);
                }
            }
        }
#pragma unroll
        for (int o = LJ_TPP / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (act && l4 == 0) b.ap_part[(size_t)js * b.np + p] = make_float4(fx, fy, fz, 0.f);
        if (ENERGY) {
            double de = 0.5 * (double)e, dw = 0.5 * (double)vir;
            block_sum2(de, dw, s_red);
            if (threadIdx.x == 0) {
                b.ap_pe[2 * (size_t)it] = de;
                b.ap_pe[2 * (size_t)it + 1] = dw;
            }
        }
        if (last_slice(b, w, &s_flag)) {
            for (int q = ch.y + (int)threadIdx.x; q < ch.z; q += blockDim.x) {
                float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int k = 0; k < b.ap_js; ++k) {
                    const float4 g = __ldcg(&b.ap_part[(size_t)k * b.np + q]);
                    f.x += g.x;
                    f.y += g.y;
                    f.z += g.z;
                }
                b.force4[q] = f;
                if (!isfinite(f.x + f.y + f.z)) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
            }
            if (ENERGY && threadIdx.x == 0) {
                double de = 0.0, dw = 0.0;
                for (int k = 0; k < b.ap_js; ++k) {
                    de += __ldcg(&b.ap_pe[2 * ((size_t)w * b.ap_js + k)]);
                    dw += __ldcg(&b.ap_pe[2 * ((size_t)w * b.ap_js + k) + 1]);
                }
                b.part_f[2 * w] = de;
                b.part_f[2 * w + 1] = dw;
            }
        }
    }
}

// All pairs in FP64 (MD_PREC_FP64): the same work items, one thread per
// particle, FP64 offsets staged through shared memory; partial forces in
// b.ap_part64 (3 planes per slice).
template <bool ENERGY>
__global__ void __launch_bounds__(LJ_CHUNK) k_force_all_f64(BoxDev b)
{
    constexpr int kT = 512;
    __shared__ double s_x[kT], s_y[kT], s_z[kT];
    __shared__ int s_t[kT];
    __shared__ double s_red[2][32];
    __shared__ int s_flag;
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    const int np = b.np;
    const int nitem = b.nchunk * b.ap_js;
    for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
        const int w = it / b.ap_js, js = it % b.ap_js;
        const int4 ch = b.chunk[w];
        const RepDev& R = b.rep[ch.x];
        if (threadIdx.x == 0 && js == 0) {
            if (w == 0) *b.any_req = 0;
            if (w == R.chunk_off) {
                b.disp_max[ch.x] = 0u;
                b.rebuild_req[ch.x] = 0;
            }
        }
        const double Lx = R.L[0], Ly = R.L[1], Lz = R.L[2];
        const double ix = 1.0 / Lx, iy = 1.0 / Ly, iz = 1.0 / Lz;
        const int p = ch.y + (int)threadIdx.x;
        const bool act = p < ch.z;
        const int pa = act ? p : ch.y;
        const double xi = b.off[pa], yi = b.off[np + pa], zi = b.off[2 * np + pa];
        const int ti = b.type[pa];
        double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0, vir = 0.0;
        int j0, j1;
        slice_range(R, js, b.ap_js, j0, j1);
        for (int t0 = j0; t0 < j1; t0 += kT) {
            const int nj = min(kT, j1 - t0);
            __syncthreads();
            for (int t = threadIdx.x; t < nj; t += blockDim.x) {
                s_x[t] = b.off[t0 + t];
                s_y[t] = b.off[np + t0 + t];
                s_z[t] = b.off[2 * np + t0 + t];
                s_t[t] = b.type[t0 + t];
            }
            __syncthreads();
            if (!act) continue;
            for (int t = 0; t < nj; ++t) {
                if (t0 + t == p) continue;
                double dx = xi - s_x[t], dy = yi - s_y[t], dz = zi - s_z[t];
                dx -= Lx * rint(dx * ix);
                dy -= Ly * rint(dy * iy);
                dz -= Lz * rint(dz * iz);
                const double r2 = dx * dx + dy * dy + dz * dz;
                const int pp = ti * nt + s_t[t];
                const double r2i = 1.0 / r2;
                const double s2 = lj->dsig2[pp] * r2i;
                const double s6 = s2 * s2 * s2;
                const double f = lj->deps48[pp] * r2i * s6 * (s6 - 0.5);
                fx += f * dx;
                fy += f * dy;
                fz += f * dz;
                if (ENERGY) {
                    e += lj->deps4[pp] * s6 * (s6 - 1.0) - lj->dshift[pp];
                    vir += f * r2;
                }
            }
        }
        if (act) {
            double* part = b.ap_part64 + (size_t)js * 3 * np;
            part[p] = fx;
            part[np + p] = fy;
            part[2 * np + p] = fz;
        }
        if (ENERGY) {
            double de = 0.5 * e, dw = 0.5 * vir;
            block_sum2(de, dw, s_red);
            if (threadIdx.x == 0) {
                b.ap_pe[2 * (size_t)it] = de;
                b.ap_pe[2 * (size_t)it + 1] = dw;
            }
        }
        if (last_slice(b, w, &s_flag)) {
            for (int q = ch.y + (int)threadIdx.x; q < ch.z; q += blockDim.x) {
                double f[3] = {0.0, 0.0, 0.0};
                for (int k = 0; k < b.ap_js; ++k)
                    for (int c = 0; c < 3; ++c) f[c] += __ldcg(&b.ap_part64[(size_t)k * 3 * np + (size_t)c * np + q]);
                for (int c = 0; c < 3; ++c) b.force64[(size_t)c * np + q] = f[c];
                if (!isfinite(f[0] + f[1] + f[2])) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
            }
            if (ENERGY && threadIdx.x == 0) {
                double de = 0.0, dw = 0.0;
                for (int k = 0; k < b.ap_js; ++k) {
                    de += __ldcg(&b.ap_pe[2 * ((size_t)w * b.ap_js + k)]);
                    dw += __ldcg(&b.ap_pe[2 * ((size_t)w * b.ap_js + k) + 1]);
                }
                b.part_f[2 * w] = de;
                b.part_f[2 * w + 1] = dw;
            }
        }
    }
}

// E_pot, E_kin, W, T per replica from the per-chunk partial sums, in a
// fixed order (deterministic): each block of LJ_THERMO_THREADS sums one item
// (a run of up to LJ_THERMO_CHUNKS chunks of one replica, pf_stride
// (E_pot, W) shares and LJ_KIN_WARPS E_kin shares per chunk).  A replica
// of one item is written out by its block directly; otherwise each block
// stores its 3 sums and the block that completes the replica's last item
// (atomic count) adds the item sums in item order and resets the count.
__global__ void __launch_bounds__(LJ_THERMO_THREADS) k_thermo(BoxDev b, double* out, int with_kin)
{
    __shared__ double s_red[3][LJ_THERMO_THREADS / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto block_sum3 = [&](double& e, double& w, double& k) {
        e = warp_sum_d(e);
        w = warp_sum_d(w);
        k = warp_sum_d(k);
        if (lane == 0) {
            s_red[0][warp] = e;
            s_red[1][warp] = w;
            s_red[2][warp] = k;
        }
        __syncthreads();
        if (warp == 0) {   // the warp sums in a fixed order: lane q holds warp q's sums
            const int nw = blockDim.x >> 5;
            e = lane < nw ? s_red[0][lane] : 0.0;
            w = lane < nw ? s_red[1][lane] : 0.0;
            k = lane < nw ? s_red[2][lane] : 0.0;
            e = warp_sum_d(e);
            w = warp_sum_d(w);
            k = warp_sum_d(k);
        }
        __syncthreads();
    };
    auto write_out = [&](const RepDev& R, int r, double e, double w, double k) {
        out[4 * r + 0] = e;
        out[4 * r + 1] = k;
        out[4 * r + 2] = w;
        out[4 * r + 3] = R.n > 1 ? 2.0 * k / (3.0 * (double)R.n - 3.0) : 0.0;
    };
    for (int it = blockIdx.x; it < b.ntitem; it += gridDim.x) {
        const int4 t = b.titem[it];
        const int r = t.x;
        const RepDev& R = b.rep[r];
        double e = 0.0, w = 0.0, k = 0.0;
        const int pf = b.pf_stride;
        const double2* sh = reinterpret_cast<const double2*>(b.part_f);   // (E_pot, W) shares
        // the item's (E_pot, W) shares: those of its chunks, or, from the
        // tiled force kernel, those of its share of the replica's bricks
        int s0 = t.y * pf, s1 = t.z * pf;
        if (b.force_tiles) {
            const int q = it - R.ti_off;
            s0 = (R.brick_off + (int)(((long long)q * R.nbrick) / R.nti)) * pf;
            s1 = (R.brick_off + (int)(((long long)(q + 1) * R.nbrick) / R.nti)) * pf;
        }
        // four independent loads in flight per thread, then their sums
        const int nt4 = 4 * (int)blockDim.x;
        for (int c0 = s0; c0 < s1; c0 += nt4) {
            double2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + u * (int)blockDim.x + (int)threadIdx.x;
                if (b.pf_ds) {   // (hi, lo) float pairs
                    const float4 f = c < s1 ? reinterpret_cast<const float4*>(b.part_f)[c]
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[u] = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
                } else {
                    v[u] = c < s1 ? sh[c] : make_double2(0.0, 0.0);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                e += v[u].x;
                w += v[u].y;
            }
        }
        if (with_kin)
            for (int c0 = t.y * LJ_KIN_WARPS; c0 < t.z * LJ_KIN_WARPS; c0 += nt4) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = c0 + u * (int)blockDim.x + (int)threadIdx.x;
                    v[u] = c < t.z * LJ_KIN_WARPS ? b.part_k[c] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) k += v[u];
            }
        block_sum3(e, w, k);
        if (R.nti == 1) {   // block-uniform: the replica's only item
            if (threadIdx.x == 0) write_out(R, r, e, w, k);
            continue;
        }
        if (threadIdx.x == 0) {
            b.part_t[3 * it + 0] = e;
            b.part_t[3 * it + 1] = w;
            b.part_t[3 * it + 2] = k;
            __threadfence();
            s_last = atomicAdd(&b.tcount[r], 1u) == (unsigned)(R.nti - 1);
        }
        __syncthreads();
        if (s_last) {   // block-uniform
            __threadfence();
            e = w = k = 0.0;
            for (int i = R.ti_off + (int)threadIdx.x; i < R.ti_off + R.nti; i += blockDim.x) {
                e += __ldcg(&b.part_t[3 * i + 0]);
                w += __ldcg(&b.part_t[3 * i + 1]);
                k += __ldcg(&b.part_t[3 * i + 2]);
            }
            block_sum3(e, w, k);
            if (threadIdx.x == 0) {
                write_out(R, r, e, w, k);
                b.tcount[r] = 0u;
            }
        }
        __syncthreads();
    }
}

}  // namespace

// The tiled force kernel's dynamic shared memory (two buffers) is above the
// default 48 KB: raise the limit once per process.
static cudaError_t tile_kernel_attrs()
{
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady) {
        cudaError_t e = cudaSuccess;
        const int dm = (int)(2 * tile_buf_bytes(true)), dx = (int)(2 * tile_buf_bytes(false));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_tile_f32<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_tile_f32<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_tile_f32<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_force_tile_f32<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dx);
        done = e;
    }
    return done;
}

cudaError_t launch_force(const BoxDev& b, int energy, Launch l)
{
    if (b.all_pairs) {
        if (b.prec == 2) {
            if (energy) k_force_all_f64<true><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
            else k_force_all_f64<false><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
        } else if (b.nt == 1) {
            if (energy) k_force_all_f32<true, true><<<l.grid, kAllThreads, 0, l.s>>>(b);
            else k_force_all_f32<true, false><<<l.grid, kAllThreads, 0, l.s>>>(b);
        } else {
            if (energy) k_force_all_f32<false, true><<<l.grid, kAllThreads, 0, l.s>>>(b);
            else k_force_all_f32<false, false><<<l.grid, kAllThreads, 0, l.s>>>(b);
        }
        return cudaGetLastError();
    }
    if (b.prec == 2) {
        if (energy) k_force_f64<true><<<l.grid, LJ_F64_THREADS, 0, l.s>>>(b);
        else k_force_f64<false><<<l.grid, LJ_F64_THREADS, 0, l.s>>>(b);
    } else if (b.force_tiles) {
        cudaError_t e = tile_kernel_attrs();
        if (e != cudaSuccess) return e;
        const int th = LJ_BRICK_THREADS + 32;
        const size_t dm = 2 * tile_buf_bytes(true), dx = 2 * tile_buf_bytes(false);
        if (b.nt == 1) {
            if (energy) k_force_tile_f32<true, true><<<l.grid, th, dm, l.s>>>(b);
            else k_force_tile_f32<true, false><<<l.grid, th, dm, l.s>>>(b);
        } else {
            if (energy) k_force_tile_f32<false, true><<<l.grid, th, dx, l.s>>>(b);
            else k_force_tile_f32<false, false><<<l.grid, th, dx, l.s>>>(b);
        }
    } else if (b.nt == 1 && b.nrep == 1) {
        if (energy) k_force_f32<true, true, true><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
        else k_force_f32<true, false, true><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
    } else if (b.nt == 1) {
        if (energy) k_force_f32<true, true, false><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
        else k_force_f32<true, false, false><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
    } else {
        if (energy) k_force_f32<false, true, false><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
        else k_force_f32<false, false, false><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b);
    }
    return cudaGetLastError();
}

// Resident blocks per SM of the tiled force kernel (its persistent grid).
int force_tile_blocks_per_sm(int mono)
{
    static int occ[2] = {0, 0};
    int& o = occ[mono ? 1 : 0];
    if (o == 0 && tile_kernel_attrs() == cudaSuccess) {
        int v = 0;
        const int th = LJ_BRICK_THREADS + 32;
        cudaError_t e = mono ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_force_tile_f32<true, true>, th,
                                                                             2 * tile_buf_bytes(true))
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_force_tile_f32<false, true>, th,
                                                                             2 * tile_buf_bytes(false));
        o = (e == cudaSuccess && v > 0) ? v : 2;
    }
    return o > 0 ? o : 2;
}

cudaError_t launch_thermo(const BoxDev& b, double* out, int with_kin, Launch l)
{
    k_thermo<<<l.grid, LJ_THERMO_THREADS, 0, l.s>>>(b, out, with_kin);
    return cudaGetLastError();
}
