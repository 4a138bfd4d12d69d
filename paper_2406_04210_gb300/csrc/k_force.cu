// k_force.cu -- truncated Lennard-Jones pair force, energy and virial over the
// Verlet list (Sec. 4: Lennard-Jones pair forces; Sec. 5, Truncated Force
// Performance Study: the force kernel over Verlet lists is ~60 % of the run
// time and is memory-latency sensitive -- the CUDA version there reads packed
// float4 particle data through the texture path).
//
// One thread per particle i, in cell-sorted order, walks its list:
//   d_ij = (o_i - o_j) - shift(k)       cell-relative offsets, FP32
//   F_i += 48 eps/r^2 [(s/r)^12 - (s/r)^6/2] d_ij      for r^2 < rc^2
// E_pot and W are summed per particle in the kernel's real type, reduced per
// work item in FP64 (each pair is seen twice in a full list: factor 1/2).
#include "ljmd_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum two doubles over the block (blockDim == LJ_CHUNK); valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& c, double (*s)[LJ_CHUNK / 32])
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
        for (int k = 0; k < LJ_CHUNK / 32; ++k) {
            a += s[0][k];
            c += s[1][k];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void load_shift_table(float4* s_shift, const RepDev& R)
{
    if (threadIdx.x < 27) {
        int k = threadIdx.x;
        s_shift[k] = make_float4((float)(k % 3 - 1) * R.ellf[0], (float)((k / 3) % 3 - 1) * R.ellf[1],
                                 (float)(k / 9 - 1) * R.ellf[2], 0.f);
    }
}

// FP32 force.  MONO: a single species, parameters in registers.
template <bool MONO, bool ENERGY>
__global__ void __launch_bounds__(LJ_CHUNK) k_force_f32(BoxDev b)
{
    __shared__ float4 s_shift[27];
    __shared__ float4 s_par[LJ_MAXT * LJ_MAXT];   // sig2, eps48, eps4, shift
    __shared__ float s_rc2[LJ_MAXT * LJ_MAXT];
    __shared__ double s_red[2][LJ_CHUNK / 32];
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) {
        s_par[k] = make_float4(lj->sig2[k], lj->eps48[k], lj->eps4[k], lj->shift[k]);
        s_rc2[k] = lj->rc2[k];
    }
    const float m_sig2 = lj->sig2[0], m_eps48 = lj->eps48[0], m_eps4 = lj->eps4[0],
                m_shift = lj->shift[0], m_rc2 = lj->rc2[0];
    int cur_r = -1;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int r = ch.x;
        const RepDev& R = b.rep[r];
        if (r != cur_r) {
            __syncthreads();
            load_shift_table(s_shift, R);
            __syncthreads();
            cur_r = r;
        }
        if (threadIdx.x == 0 && ch.y == R.p_off) {
            // the list of this replica is now used: clear the rebuild triggers
            b.disp_max[r] = 0u;
            b.rebuild_req[r] = 0;
        }
        int p = ch.y + (int)threadIdx.x;
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, vir = 0.f;
        if (p < ch.z) {
            float4 pi = b.posq[p];
            int ti = __float_as_int(pi.w);
            int cnt = min(b.nbr_count[p], b.K);
            const uint32_t* lp = b.nbr + (size_t)(p >> 5) * (size_t)b.K * 32 + (p & 31);
#pragma unroll 4
            for (int s = 0; s < cnt; ++s) {
                uint32_t ent = __ldcs(lp + (size_t)s * 32);
                int j = (int)(ent & LJ_IDX_MASK);
                float4 sh = s_shift[ent >> LJ_IDX_BITS];
                float4 pj = __ldg(&b.posq[j]);
                float dx = (pi.x - pj.x) - sh.x;
                float dy = (pi.y - pj.y) - sh.y;
                float dz = (pi.z - pj.z) - sh.z;
                float r2 = dx * dx + dy * dy + dz * dz;
                float sig2, eps48, eps4, shv, rc2;
                if (MONO) {
                    sig2 = m_sig2; eps48 = m_eps48; eps4 = m_eps4; shv = m_shift; rc2 = m_rc2;
                } else {
                    int pp = ti * nt + __float_as_int(pj.w);
                    float4 q = s_par[pp];
                    sig2 = q.x; eps48 = q.y; eps4 = q.z; shv = q.w; rc2 = s_rc2[pp];
                }
                if (r2 < rc2) {
                    float r2i = __frcp_rn(r2);
                    float s2 = sig2 * r2i;
                    float s6 = s2 * s2 * s2;
                    float f = eps48 * r2i * s6 * (s6 - 0.5f);
                    fx += f * dx;
                    fy += f * dy;
                    fz += f * dz;
                    if (ENERGY) {
                        e += eps4 * s6 * (s6 - 1.0f) - shv;
                        vir += f * r2;
                    }
                }
            }
            b.force4[p] = make_float4(fx, fy, fz, 0.f);
            if (!isfinite(fx + fy + fz)) atomicOr(&b.err[0], LJ_ERRBIT_NONFINITE);
        }
        if (ENERGY) {
            double de = 0.5 * (double)e, dw = 0.5 * (double)vir;
            block_sum2(de, dw, s_red);
            if (threadIdx.x == 0) {
                b.part_f[2 * w] = de;
                b.part_f[2 * w + 1] = dw;
            }
        }
    }
}

// FP64 force from the FP64 cell-relative offsets (MD_PREC_FP64).
template <bool ENERGY>
__global__ void __launch_bounds__(LJ_CHUNK) k_force_f64(BoxDev b)
{
    __shared__ double s_sh[3][27];
    __shared__ double s_red[2][LJ_CHUNK / 32];
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    const int np = b.np;
    int cur_r = -1;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int r = ch.x;
        const RepDev& R = b.rep[r];
        if (r != cur_r) {
            __syncthreads();
            if (threadIdx.x < 27) {
                int k = threadIdx.x;
                s_sh[0][k] = (double)(k % 3 - 1) * R.ell[0];
                s_sh[1][k] = (double)((k / 3) % 3 - 1) * R.ell[1];
                s_sh[2][k] = (double)(k / 9 - 1) * R.ell[2];
            }
            __syncthreads();
            cur_r = r;
        }
        if (threadIdx.x == 0 && ch.y == R.p_off) {
            b.disp_max[r] = 0u;
            b.rebuild_req[r] = 0;
        }
        int p = ch.y + (int)threadIdx.x;
        double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0, vir = 0.0;
        if (p < ch.z) {
            double xi = b.off[p], yi = b.off[np + p], zi = b.off[2 * np + p];
            int ti = b.type[p];
            int cnt = min(b.nbr_count[p], b.K);
            const uint32_t* lp = b.nbr + (size_t)(p >> 5) * (size_t)b.K * 32 + (p & 31);
            for (int s = 0; s < cnt; ++s) {
                uint32_t ent = __ldcs(lp + (size_t)s * 32);
                int j = (int)(ent & LJ_IDX_MASK);
                int k = (int)(ent >> LJ_IDX_BITS);
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
            double de = 0.5 * e, dw = 0.5 * vir;
            block_sum2(de, dw, s_red);
            if (threadIdx.x == 0) {
                b.part_f[2 * w] = de;
                b.part_f[2 * w + 1] = dw;
            }
        }
    }
}

// One warp per replica: E_pot, E_kin, W, T from the per-chunk partial sums,
// in a fixed order (deterministic).
__global__ void k_thermo(BoxDev b, double* out, int with_kin)
{
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < b.nrep; r += gridDim.x * wpb) {
        const RepDev& R = b.rep[r];
        double e = 0.0, w = 0.0, k = 0.0;
        for (int c = R.chunk_off + lane; c < R.chunk_off + R.nchunk; c += 32) {
            e += b.part_f[2 * c];
            w += b.part_f[2 * c + 1];
            if (with_kin) k += b.part_k[c];
        }
        e = warp_sum_d(e);
        w = warp_sum_d(w);
        k = warp_sum_d(k);
        if (lane == 0) {
            out[4 * r + 0] = e;
            out[4 * r + 1] = k;
            out[4 * r + 2] = w;
            out[4 * r + 3] = R.n > 1 ? 2.0 * k / (3.0 * (double)R.n - 3.0) : 0.0;
        }
    }
}

}  // namespace

cudaError_t launch_force(const BoxDev& b, int energy, Launch l)
{
    if (b.prec == 2) {
        if (energy) k_force_f64<true><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
        else k_force_f64<false><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
    } else {
        bool mono = b.nt == 1;
        if (mono) {
            if (energy) k_force_f32<true, true><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
            else k_force_f32<true, false><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
        } else {
            if (energy) k_force_f32<false, true><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
            else k_force_f32<false, false><<<l.grid, LJ_CHUNK, 0, l.s>>>(b);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_thermo(const BoxDev& b, double* out, int with_kin, Launch l)
{
    k_thermo<<<l.grid, 128, 0, l.s>>>(b, out, with_kin);
    return cudaGetLastError();
}
