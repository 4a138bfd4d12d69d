// k_adjoint.cu -- reverse-mode derivative of the velocity-Verlet LJ trajectory
// and the smoothed pair-distance histogram used as a trajectory loss.
//
// The paper has no adjoint; these kernels differentiate the steps of the
// integrator (Sec. 3, Fig. 1: integrate / force / finalize; unit mass):
//   forward   vh = v_k + h/2 F(x_k); x_{k+1} = x_k + h vh; v_{k+1} = vh + h/2 F(x_{k+1})
//   reverse   lx~ = lx_{k+1} - h/2 H(x_{k+1}) lv_{k+1};  lvh = lv_{k+1} + h lx~
//             lx_k = lx~ - h/2 H(x_k) lvh;  lv_k = lvh
//   with H = Hessian of U_tot, so dF/dx = -H.  H(x_k) lvh is reused as the
//   H(x_{k+1}) lv_{k+1} term of the step before: one Hessian-vector product
//   (HVP) per step.  Parameter gradients add h/2 lv . dF/dtheta at every
//   state (twice at interior states).
// Pair HVP, with d = x_i - x_j, u_ij = u_i - u_j and the cutoff held fixed:
//   (H u)_i = sum_j [A d (d . u_ij) - f u_ij],
//   f = 48 eps s^6 (s^6 - 1/2) / r^2   (force coefficient, -phi'/r)
//   A = (phi'' - phi'/r) / r^2 = 672 eps sigma^12 / r^16 - 192 eps sigma^6 / r^10
// Parameter derivatives of F_ij = f d at fixed r and rc:
//   dF/deps = (f/eps) d,  dF/dsigma = (576 eps sigma^11 / r^14 - 144 eps sigma^5 / r^8) d
#include "ljmd_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// u (user order, FP64 n x 3) -> slot order FP32 for the HVP kernel, after
// the adjoint half-update of this step:
//   pre = 1: lx <- lx - h/2 g;  lv <- lv + h lx;  u = lv   (then HVP of u)
//   pre = 0: u = lv                                         (first state)
__global__ void __launch_bounds__(LJ_CHUNK) k_adj_pre(BoxDev b, double* lx, double* lv, const double* g,
                                                      float4* u_slot, double h, int pre)
{
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        int4 ch = b.chunk[w];
        int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        size_t gu = (size_t)b.uid[p];
        float uf[3];
        for (int c = 0; c < 3; ++c) {
            double v = lv[3 * gu + c];
            if (pre) {
                double x = lx[3 * gu + c] - 0.5 * h * g[3 * gu + c];
                lx[3 * gu + c] = x;
                v = v + h * x;
                lv[3 * gu + c] = v;
            }
            uf[c] = (float)v;
        }
        u_slot[p] = make_float4(uf[0], uf[1], uf[2], 0.f);
    }
}

// HVP and parameter-gradient terms at one state, LJ_TPP threads per particle
// (as the force kernel), with the adjoint update that follows it:
//   g <- H u (user order, FP64);  lx <- lx - h/2 g   (when upd)
// part_g[chunk * 2P + 0..P-1] accumulates weight * sum lam.dF/deps and
// [P..2P-1] weight * sum lam.dF/dsigma per symmetric type pair (P = nt * nt
// slots; the (a, b) and (b, a) terms both land in the slot of min/max) over
// the states of the reverse sweep; one reduction at its end.  MONO keeps the
// two sums in registers and accumulates one pair per warp and chunk,
// part_g[(chunk * LJ_FORCE_WARPS + warp) * 2 + 0/1], with no block barrier
// (deterministic); otherwise shared-memory atomics, one 2P row per chunk.
template <bool MONO>
__global__ void __launch_bounds__(LJ_FORCE_THREADS) k_hvp_f32(BoxDev b, const float4* __restrict__ u_slot,
                                                              double* lx, double* g, double h, int upd,
                                                              const double* weight, double* part_g)
{
    __shared__ float4 s_c[LJ_MAXT * LJ_MAXT];     // c12, c6, a12, a6
    __shared__ float4 s_g[LJ_MAXT * LJ_MAXT];     // g12, g6, 1/eps, rc2
    __shared__ float s_acc[2 * LJ_MAXT * LJ_MAXT];
    const LJDev* lj = b.lj;
    const int nt = lj->nt;
    const int P = nt * nt;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        s_c[k] = make_float4(lj->c12[k], lj->c6[k], lj->a12[k], lj->a6[k]);
        s_g[k] = make_float4(lj->g12[k], lj->g6[k], lj->inv_eps[k], lj->rc2[k]);
    }
    __syncthreads();   // the pair tables are complete
    const float4 mc = make_float4(lj->c12[0], lj->c6[0], lj->a12[0], lj->a6[0]);
    const float4 mg = make_float4(lj->g12[0], lj->g6[0], lj->inv_eps[0], lj->rc2[0]);
    const int K = b.K;
    const int grp = threadIdx.x / LJ_TPP, l8 = threadIdx.x % LJ_TPP;
    const float4* __restrict__ posq = b.posq;
    int cur_r = -1;
    float3 ell = make_float3(0.f, 0.f, 0.f);
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        const int4 ch = b.chunk[w];
        const int r = ch.x;
        if (r != cur_r) {                       // block-uniform
            const RepDev& R = b.rep[r];
            ell = make_float3(R.ellf[0], R.ellf[1], R.ellf[2]);
            cur_r = r;
        }
        if (!MONO) {   // per-chunk species-pair sums in shared memory
            __syncthreads();
            for (int k = threadIdx.x; k < 2 * P; k += blockDim.x) s_acc[k] = 0.f;
            __syncthreads();
        }
        float ge = 0.f, gs = 0.f;
        for (int base = ch.y; base < ch.z; base += LJ_FORCE_THREADS / LJ_TPP) {
            const int p = base + grp;
            const bool act = p < ch.z;
            float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), ui = pi;
            int cnt = 0;
            if (act) {
                pi = posq[p];
                ui = u_slot[p];
                cnt = min(b.nbr_count[p], K);
            }
            const int ti = __float_as_int(pi.w);
            const uint32_t* L = b.nbr + (size_t)K * p;
            float hx = 0.f, hy = 0.f, hz = 0.f;
            for (int s = l8; s < cnt; s += LJ_TPP) {
                const unsigned ent = __ldcs(L + s);
                const int j = (int)(ent & LJ_IDX_MASK);
                const float4 pj = __ldg(posq + j);
                const float4 uj = __ldg(u_slot + j);
                // d = (o_i - o_j) - (dx, dy, dz) * ell, one rounding per component
                const float dx = fmaf(-entry_unit(ent, 26), ell.x, pi.x - pj.x);
                const float dy = fmaf(-entry_unit(ent, 28), ell.y, pi.y - pj.y);
                const float dz = fmaf(-entry_unit(ent, 30), ell.z, pi.z - pj.z);
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float4 c, gg;
                int pp = 0;
                if (MONO) {
                    c = mc;
                    gg = mg;
                } else {
                    pp = ti * nt + __float_as_int(pj.w);
                    c = s_c[pp];
                    gg = s_g[pp];
                }
                const bool in = r2 < gg.w;
                const float r2i = rcp_approx(r2);
                const float r6i = r2i * r2i * r2i;
                float f = r2i * r6i * fmaf(c.x, r6i, -c.y);
                float A = r2i * r2i * r6i * fmaf(c.z, r6i, -c.w);
                f = in ? f : 0.f;
                A = in ? A : 0.f;
                const float ux = ui.x - uj.x, uy = ui.y - uj.y, uz = ui.z - uj.z;
                const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
                const float Adu = A * du;
                hx = fmaf(Adu, dx, fmaf(-f, ux, hx));
                hy = fmaf(Adu, dy, fmaf(-f, uy, hy));
                hz = fmaf(Adu, dz, fmaf(-f, uz, hz));
                const float ld = fmaf(ui.x, dx, fmaf(ui.y, dy, ui.z * dz));
                const float dsg = in ? r2i * r6i * fmaf(gg.x, r6i, -gg.y) * ld : 0.f;
                const float dep = f * gg.z * ld;
                if (MONO) {
                    ge += dep;
                    gs += dsg;
                } else if (in) {
                    const int a = ti, bb = __float_as_int(pj.w);
                    const int q = (a < bb ? a : bb) * nt + (a < bb ? bb : a);
                    atomicAdd(&s_acc[q], dep);
                    atomicAdd(&s_acc[P + q], dsg);
                }
            }
#pragma unroll
            for (int o = LJ_TPP / 2; o > 0; o >>= 1) {
                hx += __shfl_xor_sync(0xffffffffu, hx, o);
                hy += __shfl_xor_sync(0xffffffffu, hy, o);
                hz += __shfl_xor_sync(0xffffffffu, hz, o);
            }
            if (act && l8 == 0) {
                const size_t gu = (size_t)b.uid[p];
                const double hv[3] = {hx, hy, hz};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    g[3 * gu + c] = hv[c];
                    if (upd) lx[3 * gu + c] = lx[3 * gu + c] - 0.5 * h * hv[c];
                }
            }
        }
        const double wgt = *weight;
        if (MONO) {
            // one (d/deps, d/dsigma) share per warp and chunk (no block barrier)
            const double de = warp_sum_ds(ge), ds = warp_sum_ds(gs);   // double-single warp sums
            if ((threadIdx.x & 31) == 0) {
                const size_t q = (size_t)w * LJ_FORCE_WARPS + (threadIdx.x >> 5);
                part_g[2 * q] += wgt * de;
                part_g[2 * q + 1] += wgt * ds;
            }
        } else {
            __syncthreads();
            for (int k = threadIdx.x; k < 2 * P; k += blockDim.x)
                part_g[2 * (size_t)P * w + k] += wgt * (double)s_acc[k];
        }
    }
}

// theta_grad[q] += weight * sum over chunks of part_g[chunk * 2P + q], in a
// fixed order (one block).
__global__ void __launch_bounds__(512) k_param_reduce(const double* part_g, int nchunk, int twoP,
                                                      const double* weight, double* theta_grad)
{
    __shared__ double s_red[512 / 32];
    const double wgt = *weight;
    for (int q = 0; q < twoP; ++q) {
        double s = 0.0;
        for (int c = threadIdx.x; c < nchunk; c += blockDim.x) s += part_g[(size_t)twoP * c + q];
        s = warp_sum_d(s);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_red[k];
            theta_grad[q] += wgt * t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Smoothed pair-distance histogram over the current list (a trajectory
// loss):  h_k = (1/N_r) sum_{i<j, r_ij < rmax} exp(-(r_ij - c_k)^2 / (2 w^2)),
// c_k = (k + 1/2) rhist / nbins, per replica (N_r its particle count).  The
// lists must have been built at the current positions with rl >= rmax, so
// that they hold every pair below rmax.  Pairs are counted once (uid_i <
// uid_j).  part_h[chunk * nbins + k]: per-chunk sums, reduced per replica.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(LJ_CHUNK) k_pair_hist(BoxDev b, int nbins, float rbin, float inv2w2,
                                                        float rmax2, double* part_h)
{
    __shared__ double s_red[LJ_CHUNK / 32];
    __shared__ float4 s_shift[32];
    int cur_r = -1;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        const int4 ch = b.chunk[w];
        __syncthreads();
        if (ch.x != cur_r && threadIdx.x < 32) {
            const RepDev& R = b.rep[ch.x];
            const int k = threadIdx.x;
            s_shift[k] = k < 27 ? make_float4((float)(k % 3 - 1) * R.ellf[0], (float)((k / 3) % 3 - 1) * R.ellf[1],
                                              (float)(k / 9 - 1) * R.ellf[2], 0.f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cur_r = ch.x;
        __syncthreads();
        const int p = ch.y + (int)threadIdx.x;
        const bool act = p < ch.z;
        float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
        int cnt = 0, ui = 0;
        if (act) {
            pi = b.posq[p];
            cnt = min(b.nbr_count[p], b.K);
            ui = b.uid[p];
        }
        const uint32_t* L = b.nbr + (size_t)b.K * p;
        for (int k = 0; k < nbins; ++k) {
            const float ck = ((float)k + 0.5f) * rbin;
            float acc = 0.f;
            for (int s = 0; s < cnt; ++s) {
                const unsigned ent = L[s];
                const int j = (int)(ent & LJ_IDX_MASK);
                if (b.uid[j] <= ui) continue;
                const float4 pj = b.posq[j];
                const float4 sh = s_shift[entry_k(ent)];
                const float dx = (pi.x - pj.x) - sh.x, dy = (pi.y - pj.y) - sh.y, dz = (pi.z - pj.z) - sh.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rmax2)) continue;
                const float dr = sqrtf(r2) - ck;
                acc += __expf(-dr * dr * inv2w2);
            }
            double t = warp_sum_d((double)acc);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double q = 0.0;
                for (int m = 0; m < LJ_CHUNK / 32; ++m) q += s_red[m];
                part_h[(size_t)w * nbins + k] = q;
            }
            __syncthreads();
        }
    }
}

// per-replica histogram from the chunk sums: h[r * nbins + k] = sum / n_r
__global__ void k_hist_reduce(BoxDev b, int nbins, const double* part_h, double* h)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < b.nrep * nbins; idx += gridDim.x * blockDim.x) {
        const int r = idx / nbins, k = idx % nbins;
        const RepDev& R = b.rep[r];
        double s = 0.0;
        for (int c = R.chunk_off; c < R.chunk_off + R.nchunk; ++c) s += part_h[(size_t)c * nbins + k];
        h[idx] = R.n > 0 ? s / (double)R.n : 0.0;
    }
}

// gradient of sum_k coef[r, k] h_{r,k} with respect to the positions (user
// order, FP64): dh_k/dx_i = (1/N_r) sum_j g_k'(r_ij) d_ij / r_ij over i's
// full list (every pair seen from both ends), g_k' = -(r - c_k)/w^2 g_k.
__global__ void __launch_bounds__(LJ_CHUNK) k_pair_hist_grad(BoxDev b, int nbins, float rbin, float inv2w2,
                                                             float inv_w2, float rmax2, const double* coef,
                                                             double* grad)
{
    __shared__ float4 s_shift[32];
    __shared__ float s_coef[256];
    int cur_r = -1;
    for (int w = blockIdx.x; w < b.nchunk; w += gridDim.x) {
        const int4 ch = b.chunk[w];
        __syncthreads();
        if (ch.x != cur_r) {
            const RepDev& R = b.rep[ch.x];
            if (threadIdx.x < 32) {
                const int k = threadIdx.x;
                s_shift[k] = k < 27 ? make_float4((float)(k % 3 - 1) * R.ellf[0], (float)((k / 3) % 3 - 1) * R.ellf[1],
                                                  (float)(k / 9 - 1) * R.ellf[2], 0.f)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            for (int k = threadIdx.x; k < nbins; k += blockDim.x)
                s_coef[k] = (float)(coef[(size_t)ch.x * nbins + k] / (R.n > 0 ? (double)R.n : 1.0));
        }
        cur_r = ch.x;
        __syncthreads();
        const int p = ch.y + (int)threadIdx.x;
        if (p >= ch.z) continue;
        const float4 pi = b.posq[p];
        const int cnt = min(b.nbr_count[p], b.K);
        const uint32_t* L = b.nbr + (size_t)b.K * p;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int s = 0; s < cnt; ++s) {
            const unsigned ent = L[s];
            const int j = (int)(ent & LJ_IDX_MASK);
            const float4 pj = b.posq[j];
            const float4 sh = s_shift[entry_k(ent)];
            const float dx = (pi.x - pj.x) - sh.x, dy = (pi.y - pj.y) - sh.y, dz = (pi.z - pj.z) - sh.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rmax2)) continue;
            const float r = sqrtf(r2);
            float dg = 0.f;
            for (int k = 0; k < nbins; ++k) {
                const float dr = r - ((float)k + 0.5f) * rbin;
                dg = fmaf(s_coef[k] * (-dr * inv_w2), __expf(-dr * dr * inv2w2), dg);
            }
            const float t = dg / r;
            gx = fmaf(t, dx, gx);
            gy = fmaf(t, dy, gy);
            gz = fmaf(t, dz, gz);
        }
        const size_t gu = (size_t)b.uid[p];
        grad[3 * gu + 0] = gx;
        grad[3 * gu + 1] = gy;
        grad[3 * gu + 2] = gz;
    }
}

}  // namespace

cudaError_t launch_adj_pre(const BoxDev& b, double* lx, double* lv, const double* g, float4* u_slot, double h,
                           int pre, Launch l)
{
    k_adj_pre<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, lx, lv, g, u_slot, h, pre);
    return cudaGetLastError();
}

cudaError_t launch_hvp(const BoxDev& b, const float4* u_slot, double* lx, double* g, double h, int upd,
                       const double* weight, double* part_g, Launch l)
{
    if (b.nt == 1) k_hvp_f32<true><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b, u_slot, lx, g, h, upd, weight, part_g);
    else k_hvp_f32<false><<<l.grid, LJ_FORCE_THREADS, 0, l.s>>>(b, u_slot, lx, g, h, upd, weight, part_g);
    return cudaGetLastError();
}

cudaError_t launch_param_reduce(const double* part_g, int nchunk, int twoP, const double* weight,
                                double* theta_grad, cudaStream_t s)
{
    k_param_reduce<<<1, 512, 0, s>>>(part_g, nchunk, twoP, weight, theta_grad);
    return cudaGetLastError();
}

cudaError_t launch_pair_hist(const BoxDev& b, int nbins, double rhist, double width, double rmax, double* part_h,
                             double* h, Launch l)
{
    float rbin = (float)(rhist / nbins);
    float inv2w2 = (float)(1.0 / (2.0 * width * width));
    k_pair_hist<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, nbins, rbin, inv2w2, (float)(rmax * rmax), part_h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int n = b.nrep * nbins;
    k_hist_reduce<<<(n + 255) / 256, 256, 0, l.s>>>(b, nbins, part_h, h);
    return cudaGetLastError();
}

cudaError_t launch_pair_hist_grad(const BoxDev& b, int nbins, double rhist, double width, double rmax,
                                  const double* coef, double* grad, Launch l)
{
    float rbin = (float)(rhist / nbins);
    float inv2w2 = (float)(1.0 / (2.0 * width * width));
    float inv_w2 = (float)(1.0 / (width * width));
    k_pair_hist_grad<<<l.grid, LJ_CHUNK, 0, l.s>>>(b, nbins, rbin, inv2w2, inv_w2, (float)(rmax * rmax), coef,
                                                   grad);
    return cudaGetLastError();
}
