// k_integrate.cu -- velocity-Verlet half steps and state transfer kernels.
//
// Sec. 3 (Code structure, Fig. 1): the integrator module's `integrate`
// (half kick + drift) and `finalize` (half kick) slots run around the force
// evaluation.  The finalize of step s and the integrate of step s+1 touch the
// same particle data back to back, so LJ_STEP_MID fuses them into one pass
// (the arithmetic is unchanged: two separate half kicks, same roundings).
//
// Accumulation type ACC: 0 = double-single (two FP32 words; HAL's MD "mixed
// precision", Sec. 3), 1 = FP64.  FORCE64 selects FP64 forces.
// Per particle and step the kernel also measures the displacement since the
// last list build (FP32, from the cell-relative copies) and raises the
// replica's rebuild trigger when it exceeds skin/2 (Sec. 5: rebuilds become
// more frequent at higher temperature).
#include "ljmd_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Andersen-like collision of particle p after the finalize of step `step`
// (see md_set_thermostat): true and the new velocity in g when word 0 of
// philox((local user index, step lo, step hi, 0), seed + replica) is below
// the threshold; Gaussians by Box-Muller.
__device__ __forceinline__ bool tstat_collide(const BoxDev& b, const RepDev& R, int r, int p, long long step,
                                              double g[3])
{
    const unsigned u = (unsigned)(b.uid[p] - R.u_off);
    const unsigned long long key = b.tstat_seed + (unsigned long long)r;
    const uint2 k = make_uint2((unsigned)key, (unsigned)(key >> 32));
    const unsigned slo = (unsigned)step, shi = (unsigned)((unsigned long long)step >> 32);
    const uint4 x = philox4x32_10(make_uint4(u, slo, shi, 0u), k);
    if (!(x.x < b.tstat_thr)) return false;
    const uint4 y = philox4x32_10(make_uint4(u, slo, shi, 1u), k);
    const double sd = sqrt(b.tstat_T[r]);
    const double two_pi = 6.283185307179586476925286766559;
    const double inv32 = 1.0 / 4294967296.0;
    const double r1 = sqrt(-2.0 * log(((double)x.y + 0.5) * inv32)), a1 = two_pi * (((double)x.z + 0.5) * inv32);
    const double r2 = sqrt(-2.0 * log(((double)y.x + 0.5) * inv32)), a2 = two_pi * (((double)y.y + 0.5) * inv32);
    g[0] = sd * (r1 * cos(a1));
    g[1] = sd * (r1 * sin(a1));
    g[2] = sd * (r2 * cos(a2));
    return true;
}

// The all-pairs form (one cell per replica, offsets from the box centre):
// the drift keeps each offset in [-L/2, L/2) itself, counting the image, so
// the form needs no re-binning between steps (there are no lists).
__device__ __forceinline__ void wrap_ds(const BoxDev& b, const RepDev& R, int c, int p, float& oh, float& ol)
{
    const float lh = (float)R.L[c], ll = (float)(R.L[c] - (double)lh);
    if (oh >= 0.5f * lh) {
        ds_add_ds(oh, ol, -lh, -ll);
        b.img[c * b.np + p] += 1;
    } else if (oh < -0.5f * lh) {
        ds_add_ds(oh, ol, lh, ll);
        b.img[c * b.np + p] -= 1;
    }
}
__device__ __forceinline__ void wrap_d(const BoxDev& b, const RepDev& R, int c, int p, double& x)
{
    if (x >= 0.5 * R.L[c]) {
        x -= R.L[c];
        b.img[c * b.np + p] += 1;
    } else if (x < -0.5 * R.L[c]) {
        x += R.L[c];
        b.img[c * b.np + p] -= 1;
    }
}

// sidx: this launch finalizes step (*b.step_ctr + sidx) (MID and LAST modes).
template <int ACC, bool FORCE64, int MODE, bool ENERGY, bool TSTAT>
__global__ void __launch_bounds__(LJ_CHUNK) k_integrate(BoxDev b, double dt, int sidx)
{
    const int np = b.np;
    const double hdt = 0.5 * dt;
    float dt_h, dt_l;
    ds_from_double(dt, dt_h, dt_l);
    const float hdt_f = (float)hdt;
    float* offf = reinterpret_cast<float*>(b.off);
    float* velf = reinterpret_cast<float*>(b.vel);
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int r = ch.x;
        int p = ch.y + (int)threadIdx.x;
        double ek = 0.0;
        float ekf = 0.f;   // double-single state: FP32 per particle
        unsigned dmax = 0u;
        if (p < ch.z) {
            double F[3];
            if (FORCE64) {
                F[0] = b.force64[p];
                F[1] = b.force64[np + p];
                F[2] = b.force64[2 * np + p];
            } else {
                float4 f4 = b.force4[p];
                F[0] = f4.x;
                F[1] = f4.y;
                F[2] = f4.z;
            }
            float o[3];
            // thermostat collision after the finalize of this step
            double g[3] = {0.0, 0.0, 0.0};
            bool hit = false;
            if (TSTAT && MODE != LJ_STEP_FIRST)
                hit = tstat_collide(b, b.rep[r], r, p, *b.step_ctr + sidx, g);
            if (ACC == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float vh = velf[c * np + p], vl = velf[3 * np + c * np + p];
                    float inc = hdt_f * (float)F[c];
                    if (MODE != LJ_STEP_FIRST) {
                        ds_add_f(vh, vl, inc);
                        if (hit) ds_from_double(g[c], vh, vl);
                        if (ENERGY) ekf += vh * vh;
                    }
                    if (MODE != LJ_STEP_LAST) {
                        ds_add_f(vh, vl, inc);
                        float oh = offf[c * np + p], ol = offf[3 * np + c * np + p];
                        float ph, pl;
                        ds_mul_ds(dt_h, dt_l, vh, vl, ph, pl);
                        ds_add_ds(oh, ol, ph, pl);
                        if (b.all_pairs) wrap_ds(b, b.rep[r], c, p, oh, ol);
                        offf[c * np + p] = oh;
                        offf[3 * np + c * np + p] = ol;
                        o[c] = oh;
                    }
                    velf[c * np + p] = vh;
                    velf[3 * np + c * np + p] = vl;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double v = b.vel[c * np + p];
                    if (MODE != LJ_STEP_FIRST) {
                        v = v + hdt * F[c];
                        if (hit) v = g[c];
                        if (ENERGY) ek += v * v;
                    }
                    if (MODE != LJ_STEP_LAST) {
                        v = v + hdt * F[c];
                        double x = b.off[c * np + p] + dt * v;
                        if (b.all_pairs) wrap_d(b, b.rep[r], c, p, x);
                        b.off[c * np + p] = x;
                        o[c] = __double2float_rn(x);
                    }
                    b.vel[c * np + p] = v;
                }
            }
            if (MODE != LJ_STEP_LAST && b.all_pairs) {
                b.posq[p] = make_float4(o[0], o[1], o[2], __int_as_float(b.type[p]));
            } else if (MODE != LJ_STEP_LAST) {
                float4 rf = b.ref[p];
                b.posq[p] = make_float4(o[0], o[1], o[2], __int_as_float(b.type[p]));
                float ddx = o[0] - rf.x, ddy = o[1] - rf.y, ddz = o[2] - rf.z;
                float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                if (!(d2 <= 3.0e38f)) d2 = 3.0e38f;   // NaN or inf: force a rebuild
                dmax = __float_as_uint(d2);
            }
        }
        if (MODE != LJ_STEP_LAST) {
            unsigned m = __reduce_max_sync(0xffffffffu, dmax);
            if ((threadIdx.x & 31) == 0 && __uint_as_float(m) > b.disp_thr2) {
                atomicMax(&b.disp_max[r], m);
                atomicOr(b.any_req, 1);
            }
        }
        if (ENERGY && MODE != LJ_STEP_FIRST) {
            // one E_kin share per warp and chunk (no block barrier); the
            // double-single state sums its FP32 squares in double-single
            const double s = ACC == 0 ? 0.5 * warp_sum_ds(ekf) : warp_sum_d(0.5 * ek);
            if ((threadIdx.x & 31) == 0) b.part_k[(size_t)w * LJ_KIN_WARPS + (threadIdx.x >> 5)] = s;
        }
    }
}

template <int ACC, bool FORCE64>
cudaError_t launch_integrate_t(const BoxDev& b, int mode, int energy, double dt, int sidx, Launch l)
{
#define LJ_INT_CASE(M, E)                                                                       \
    do {                                                                                        \
        if (b.tstat_thr) k_integrate<ACC, FORCE64, M, E, true><<<l.grid, LJ_CHUNK, 0, l.s>>>(b, dt, sidx);  \
        else k_integrate<ACC, FORCE64, M, E, false><<<l.grid, LJ_CHUNK, 0, l.s>>>(b, dt, sidx);            \
    } while (0)
    if (mode == LJ_STEP_FIRST) LJ_INT_CASE(LJ_STEP_FIRST, false);
    else if (mode == LJ_STEP_MID) {
        if (energy) LJ_INT_CASE(LJ_STEP_MID, true);
        else LJ_INT_CASE(LJ_STEP_MID, false);
    } else {
        if (energy) LJ_INT_CASE(LJ_STEP_LAST, true);
        else LJ_INT_CASE(LJ_STEP_LAST, false);
    }
#undef LJ_INT_CASE
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State transfer.  User-order arrays (n x 3 FP64 AoS, device memory) <->
// the box's slot arrays.  Before the first build, slot p of replica r holds
// user particle u_off + (p - p_off).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LJ_CHUNK) k_upload(BoxDev b, const double* pos,
                                                     const double* vel, const int* type,
                                                     int set_vel)
{
    const int np = b.np;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        const RepDev& R = b.rep[ch.x];
        int gu = R.u_off + (p - R.p_off);
        for (int c = 0; c < 3; ++c) {
            double x = pos[3 * (size_t)gu + c];
            double L = R.L[c];
            double f = floor(x / L);
            b.xabs[c * np + p] = x - L * f;
            b.img[c * np + p] = (int)f;
            if (set_vel) {
                double v = vel ? vel[3 * (size_t)gu + c] : 0.0;
                if (b.prec == 0) {
                    float h, lo;
                    ds_from_double(v, h, lo);
                    float* vf = reinterpret_cast<float*>(b.vel);
                    vf[c * np + p] = h;
                    vf[3 * np + c * np + p] = lo;
                } else {
                    b.vel[c * np + p] = v;
                }
            }
        }
        b.uid[p] = gu;
        if (type) b.type[p] = type[gu];
    }
}

// Current positions (wrapped into [0, L), image counts adjusted), velocities.
__global__ void __launch_bounds__(LJ_CHUNK) k_download(BoxDev b, double* pos, double* vel,
                                                       int* img)
{
    const int np = b.np;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        const RepDev& R = b.rep[ch.x];
        int gu = b.uid[p];
        int local = b.cell[p] - R.cell_off;
        int cc[3];
        cc[0] = local % R.nc[0];
        cc[1] = (local / R.nc[0]) % R.nc[1];
        cc[2] = local / (R.nc[0] * R.nc[1]);
        for (int c = 0; c < 3; ++c) {
            double o, v;
            if (b.prec == 0) {
                const float* of = reinterpret_cast<const float*>(b.off);
                const float* vf = reinterpret_cast<const float*>(b.vel);
                o = (double)of[c * np + p] + (double)of[3 * np + c * np + p];
                v = (double)vf[c * np + p] + (double)vf[3 * np + c * np + p];
            } else {
                o = b.off[c * np + p];
                v = b.vel[c * np + p];
            }
            double x = ((double)cc[c] + 0.5) * R.ell[c] + o;
            int im = b.img[c * np + p];
            double L = R.L[c];
            double f = floor(x / L);
            if (f != 0.0) {
                x = x - L * f;
                im += (int)f;
            }
            if (pos) pos[3 * (size_t)gu + c] = x;
            if (vel) vel[3 * (size_t)gu + c] = v;
            if (img) img[3 * (size_t)gu + c] = im;
        }
    }
}

__global__ void __launch_bounds__(LJ_CHUNK) k_force_out(BoxDev b, double* f)
{
    const int np = b.np;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        size_t gu = (size_t)b.uid[p];
        if (b.prec == 2) {
            for (int c = 0; c < 3; ++c) f[3 * gu + c] = b.force64[c * np + p];
        } else {
            float4 q = b.force4[p];
            f[3 * gu + 0] = q.x;
            f[3 * gu + 1] = q.y;
            f[3 * gu + 2] = q.z;
        }
    }
}

__global__ void __launch_bounds__(LJ_CHUNK) k_get_nlist(BoxDev b, int* count, long long* nbr,
                                                        long long cap, double* pos)
{
    const int np = b.np;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        long long gu = b.uid[p];
        int cnt = b.nbr_count[p];
        count[gu] = cnt;
        if (pos)
            for (int c = 0; c < 3; ++c) pos[3 * gu + c] = b.xabs[c * np + p];
        if (nbr) {
            int m = cnt < b.K ? cnt : b.K;
            if ((long long)m > cap) m = (int)cap;
            const uint32_t* lp = b.nbr + (size_t)b.K * p;
            for (int s = 0; s < m; ++s) nbr[gu * cap + s] = b.uid[lp[s] & LJ_IDX_MASK];
        }
    }
}

}  // namespace

cudaError_t launch_integrate(const BoxDev& b, int mode, int energy, double dt, int sidx, Launch l)
{
    if (b.prec == 0) return launch_integrate_t<0, false>(b, mode, energy, dt, sidx, l);
    if (b.prec == 1) return launch_integrate_t<1, false>(b, mode, energy, dt, sidx, l);
    return launch_integrate_t<1, true>(b, mode, energy, dt, sidx, l);
}

namespace {
__global__ void k_step_advance(long long* ctr, long long n)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctr += n;
}
}  // namespace

cudaError_t launch_step_advance(long long* ctr, long long n, cudaStream_t s)
{
    k_step_advance<<<1, 32, 0, s>>>(ctr, n);
    return cudaGetLastError();
}

cudaError_t launch_upload(const BoxDev& b, const double* pos, const double* vel, const int* type,
                          int set_vel, Launch l)
{
    k_upload<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, pos, vel, type, set_vel);
    return cudaGetLastError();
}

cudaError_t launch_download(const BoxDev& b, double* pos, double* vel, int* img, Launch l)
{
    k_download<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, pos, vel, img);
    return cudaGetLastError();
}

cudaError_t launch_force_out(const BoxDev& b, double* f, Launch l)
{
    k_force_out<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, f);
    return cudaGetLastError();
}

cudaError_t launch_get_nlist(const BoxDev& b, int* count, long long* nbr, long long cap,
                             double* pos, Launch l)
{
    k_get_nlist<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, count, nbr, cap, pos);
    return cudaGetLastError();
}

namespace {
// Positions from (cell, offset) into xabs/img in place (wrapped), before the
// cell grid is changed.
__global__ void __launch_bounds__(LJ_CHUNK) k_materialize(BoxDev b)
{
    const int np = b.np;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        const RepDev& R = b.rep[ch.x];
        int local = b.cell[p] - R.cell_off;
        int cc[3];
        cc[0] = local % R.nc[0];
        cc[1] = (local / R.nc[0]) % R.nc[1];
        cc[2] = local / (R.nc[0] * R.nc[1]);
        for (int c = 0; c < 3; ++c) {
            double o;
            if (b.prec == 0) {
                const float* of = reinterpret_cast<const float*>(b.off);
                o = (double)of[c * np + p] + (double)of[3 * np + c * np + p];
            } else {
                o = b.off[c * np + p];
            }
            double x = ((double)cc[c] + 0.5) * R.ell[c] + o;
            double L = R.L[c];
            double f = floor(x / L);
            int im = b.img[c * np + p];
            if (f != 0.0) {
                x = x - L * f;
                im += (int)f;
            }
            b.xabs[c * np + p] = x;
            b.img[c * np + p] = im;
        }
    }
}
}  // namespace

cudaError_t launch_materialize(const BoxDev& b, Launch l)
{
    k_materialize<<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
    return cudaGetLastError();
}
