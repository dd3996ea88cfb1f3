// k_pair.cu -- SOG short-range pair forces, energy and virial over cell lists
// (paper sec. 2.2 and 3.1; eqs. force_SOG, U_short, P_short) plus a 12-6
// Lennard-Jones term cut (unshifted) at r_c.
//
// Per pair with r < r_c and different molecule ids:
//   f   = ke q_i q_j (1/r^3 - sum_{l<M} w~_l e^{-r^2/s~_l^2}) r_vec   (kernel N~)
//   U  += ke q_i q_j (1/r   - sum_{l<ME} w_l e^{-r^2/s_l^2})          (kernel N)
//   W  += f (x) r_vec  (eq. P_short: P^N = W / V)
// Full pairs: each atom sums all its neighbours itself (no atomics, so results
// do not depend on scheduling); energies and virials take half.
//
// Work item = one warp = a group of up to 32 atoms of one cell (lane = atom,
// in registers).  The warp walks the (2 sub + 1)^3 neighbour cells; candidate
// neighbours are read with warp-broadcast loads (every lane the same address,
// served by L1), four at a time.  A candidate that passes the cheap test
// (r^2 < r_c^2, different molecule) is pushed, with the code of its
// neighbour cell, into the lane's queue in shared memory; the warp evaluates
// the 11-transcendental SOG kernel in rounds in which every lane with an atom
// has a queued hit, so the expensive part runs with full lanes.
//
// Coordinates are cell-local (FP32 keeps ~1e-6 A); a neighbour cell's
// periodic offset (d_a w_a) is subtracted from the i coordinate.
#include "internal.h"

namespace rbsog {

namespace {

constexpr int QCAP = 64;    // per-lane queue (power of two); pending <= 32 before a batch
constexpr int WPB = 4;      // warps (work items) per block
constexpr int kMaxNb = 128; // neighbour cells of the stencil (125 for cells of r_c/2)

size_t pair_smem(int precision)
{
    return (size_t)WPB * (QCAP * 32 * (sizeof(unsigned) + 1) + kMaxNb * (precision == 1 ? 16 : 32));
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

struct AccF {
    float fx, fy, fz;
    float uc, ul, cuc, cul;   // energies with compensation terms
    float wc[6], wl[6];
};

struct AccD {
    double fx, fy, fz;
    double uc, ul;
    double wc[6], wl[6];
};

template <int NG>
__device__ __forceinline__ void pair_eval(const PairConstsF &pc, float dx, float dy, float dz, float qi,
                                          int ti, float2 qj, AccF &acc)
{
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = rsqrtf(r2);
    const float r2inv = rinv * rinv;
    float st = 0.f, se = 0.f;
    if (NG > 0) {
#pragma unroll
        for (int l = 0; l < NG; ++l) {
            float e = ex2f(-r2 * pc.beta[l]);
            st = fmaf(pc.wt[l], e, st);
            se = fmaf(pc.w[l], e, se);
        }
    } else {
        for (int l = 0; l < pc.M; ++l) {
            float e = ex2f(-r2 * pc.beta[l]);
            st = fmaf(pc.wt[l], e, st);
            se = fmaf(pc.w[l], e, se);
        }
    }
    for (int l = pc.M; l < pc.ME; ++l) se = fmaf(pc.w[l], ex2f(-r2 * pc.beta[l]), se);
    const float qq = pc.ke * qi * qj.x;
    const float fc = qq * (r2inv * rinv - st);
    const float ec = qq * (rinv - se);
    const int tj = __float_as_int(qj.y);
    const float la = pc.lj_a[ti * pc.ntypes + tj], lb = pc.lj_b[ti * pc.ntypes + tj];
    const float r6inv = r2inv * r2inv * r2inv;
    const float fl = (12.f * la * r6inv - 6.f * lb) * r6inv * r2inv;
    const float el = (la * r6inv - lb) * r6inv;
    const float f = fc + fl;
    acc.fx = fmaf(f, dx, acc.fx);
    acc.fy = fmaf(f, dy, acc.fy);
    acc.fz = fmaf(f, dz, acc.fz);
    kahan_add(acc.uc, acc.cuc, ec);
    kahan_add(acc.ul, acc.cul, el);
    const float cx = fc * dx, cy = fc * dy, lx = fl * dx, ly = fl * dy;
    acc.wc[0] = fmaf(cx, dx, acc.wc[0]); acc.wc[1] = fmaf(cy, dy, acc.wc[1]);
    acc.wc[2] = fmaf(fc * dz, dz, acc.wc[2]); acc.wc[3] = fmaf(cx, dy, acc.wc[3]);
    acc.wc[4] = fmaf(cx, dz, acc.wc[4]); acc.wc[5] = fmaf(cy, dz, acc.wc[5]);
    acc.wl[0] = fmaf(lx, dx, acc.wl[0]); acc.wl[1] = fmaf(ly, dy, acc.wl[1]);
    acc.wl[2] = fmaf(fl * dz, dz, acc.wl[2]); acc.wl[3] = fmaf(lx, dy, acc.wl[3]);
    acc.wl[4] = fmaf(lx, dz, acc.wl[4]); acc.wl[5] = fmaf(ly, dz, acc.wl[5]);
}

__device__ __forceinline__ void pair_eval(const PairConstsD &pc, double dx, double dy, double dz, double qi,
                                          int ti, double qj, int tj, AccD &acc)
{
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rinv = rsqrt(r2);
    const double r2inv = rinv * rinv;
    double st = 0.0, se = 0.0;
    for (int l = 0; l < pc.M; ++l) {
        double e = exp(-r2 * pc.inv_s2[l]);
        st = fma(pc.wt[l], e, st);
        se = fma(pc.w[l], e, se);
    }
    for (int l = pc.M; l < pc.ME; ++l) se = fma(pc.w[l], exp(-r2 * pc.inv_s2[l]), se);
    const double qq = pc.ke * qi * qj;
    const double fc = qq * (r2inv * rinv - st);
    const double ec = qq * (rinv - se);
    const double la = pc.lj_a[ti * pc.ntypes + tj], lb = pc.lj_b[ti * pc.ntypes + tj];
    const double r6inv = r2inv * r2inv * r2inv;
    const double fl = (12.0 * la * r6inv - 6.0 * lb) * r6inv * r2inv;
    const double el = (la * r6inv - lb) * r6inv;
    const double f = fc + fl;
    acc.fx = fma(f, dx, acc.fx);
    acc.fy = fma(f, dy, acc.fy);
    acc.fz = fma(f, dz, acc.fz);
    acc.uc += ec;
    acc.ul += el;
    acc.wc[0] += fc * dx * dx; acc.wc[1] += fc * dy * dy; acc.wc[2] += fc * dz * dz;
    acc.wc[3] += fc * dx * dy; acc.wc[4] += fc * dx * dz; acc.wc[5] += fc * dy * dz;
    acc.wl[0] += fl * dx * dx; acc.wl[1] += fl * dy * dy; acc.wl[2] += fl * dz * dz;
    acc.wl[3] += fl * dx * dy; acc.wl[4] += fl * dx * dz; acc.wl[5] += fl * dy * dz;
}

__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

}  // namespace

// ---------------------------------------------------------------------------
// FP32 kernel.  A queued hit carries its neighbour-cell index nb (< 125); the
// warp keeps the offsets of the (2 sub + 1)^3 neighbour cells in shared memory.
// ---------------------------------------------------------------------------
template <int NG>
__global__ void __launch_bounds__(32 * WPB)
k_pair_f32(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
           const int *__restrict__ count, const int2 *__restrict__ items, int n_items,
           const float4 *__restrict__ pos4, const float2 *__restrict__ qt, const int *__restrict__ sidx, int sub,
           double *__restrict__ F, double *__restrict__ partial, const PairConstsF pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    unsigned *q = reinterpret_cast<unsigned *>(smem) + warp * QCAP * 32;
    float4 *off = reinterpret_cast<float4 *>(smem + WPB * QCAP * 32 * sizeof(unsigned)) + warp * kMaxNb;
    unsigned char *qc = smem + WPB * QCAP * 32 * sizeof(unsigned) + WPB * kMaxNb * sizeof(float4) + warp * QCAP * 32;
    const int it = blockIdx.x * WPB + warp;
    if (it >= n_items) return;
    const int2 item = items[it];
    if (item.x < 0) return;
    const int gc = item.x;
    const DevSys &d = sys[cell_sys[gc]];
    const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
    const int lc = gc - d.cell0;
    const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
    const float wx = (float)d.w[0], wy = (float)d.w[1], wz = (float)d.w[2];
    const int span = 2 * sub + 1;
    for (int nb = lane; nb < span * span * span; nb += 32)
        off[nb] = make_float4((nb % span - sub) * wx, ((nb / span) % span - sub) * wy,
                              (nb / (span * span) - sub) * wz, 0.f);
    __syncwarp();
    const int i0 = start[gc] + 32 * item.y;
    const int ni = min(32, count[gc] - 32 * item.y);
    const bool vi = lane < ni;
    float4 pi = make_float4(0.f, 0.f, 0.f, __int_as_float(-0x7fffffff));
    float2 pq = make_float2(0.f, 0.f);
    if (vi) { pi = pos4[i0 + lane]; pq = qt[i0 + lane]; }
    const int moli = vi ? __float_as_int(pi.w) : -0x7fffffff;
    const int ti = __float_as_int(pq.y);
    const float rc2 = pc.rc2;
    AccF acc;
    acc.fx = acc.fy = acc.fz = 0.f;
    acc.uc = acc.ul = acc.cuc = acc.cul = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.wc[k] = acc.wl[k] = 0.f;
    int head = 0, tail = 0;

    auto eval_one = [&](unsigned j, int code) {
        const float4 pj = pos4[j];
        const float2 qj = qt[j];
        const float4 o = off[code];
        pair_eval<NG>(pc, (pi.x - o.x) - pj.x, (pi.y - o.y) - pj.y, (pi.z - o.z) - pj.z, pq.x, ti, qj, acc);
    };

    for (int nb = 0; nb < span * span * span; ++nb) {
        const int ddx = nb % span - sub, ddy = (nb / span) % span - sub, ddz = nb / (span * span) - sub;
        const int g = d.cell0 + wrapi(cx + ddx, n0) + n0 * (wrapi(cy + ddy, n1) + n1 * wrapi(cz + ddz, n2));
        const int j0 = start[g], nj = count[g];
        const int code = nb;
        const float4 o = off[nb];
        const float xi = pi.x - o.x, yi = pi.y - o.y, zi = pi.z - o.z;
        for (int jb = 0; jb < nj; jb += 32) {
            const int je = min(jb + 32, nj);
            int j = jb;
            for (; j + 4 <= je; j += 4) {
                float4 p[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) p[u] = __ldg(&pos4[j0 + j + u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float dx = xi - p[u].x, dy = yi - p[u].y, dz = zi - p[u].z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (vi && r2 < rc2 && __float_as_int(p[u].w) != moli) {
                        const int slot = (tail & (QCAP - 1)) * 32 + lane;
                        q[slot] = (unsigned)(j0 + j + u);
                        qc[slot] = (unsigned char)code;
                        ++tail;
                    }
                }
            }
            for (; j < je; ++j) {
                const float4 pj = __ldg(&pos4[j0 + j]);
                const float dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (vi && r2 < rc2 && __float_as_int(pj.w) != moli) {
                    const int slot = (tail & (QCAP - 1)) * 32 + lane;
                    q[slot] = (unsigned)(j0 + j);
                    qc[slot] = (unsigned char)code;
                    ++tail;
                }
            }
            // full-warp rounds: every lane with an atom has a hit queued (lanes
            // without an atom never queue anything and sit these rounds out)
            const int mn = __reduce_min_sync(0xffffffffu, vi ? tail - head : QCAP);
            for (int t = 0; t < mn; ++t) {
                if (vi) {
                    const int slot = (head & (QCAP - 1)) * 32 + lane;
                    ++head;
                    eval_one(q[slot], qc[slot]);
                }
            }
            // keep room for the next batch of 32 candidates
            while (__reduce_max_sync(0xffffffffu, tail - head) > QCAP - 32) {
                if (tail > head) {
                    const int slot = (head & (QCAP - 1)) * 32 + lane;
                    ++head;
                    eval_one(q[slot], qc[slot]);
                }
            }
        }
    }
    while (__any_sync(0xffffffffu, tail > head)) {
        if (tail > head) {
            const int slot = (head & (QCAP - 1)) * 32 + lane;
            ++head;
            eval_one(q[slot], qc[slot]);
        }
    }
    if (vi) {
        const int ia = sidx[i0 + lane];
        F[3 * ia] = acc.fx;
        F[3 * ia + 1] = acc.fy;
        F[3 * ia + 2] = acc.fz;
    }
    // per-item sums: energies in FP64 (compensated lanes), virials FP32 warp sums
    const double u0 = warp_sum((double)acc.uc - (double)acc.cuc);
    const double u1 = warp_sum((double)acc.ul - (double)acc.cul);
    float wv[12] = {acc.wc[0], acc.wc[1], acc.wc[2], acc.wc[3], acc.wc[4], acc.wc[5],
                    acc.wl[0], acc.wl[1], acc.wl[2], acc.wl[3], acc.wl[4], acc.wl[5]};
#pragma unroll
    for (int k = 0; k < 12; ++k) wv[k] = warp_sumf(wv[k]);
    if (lane == 0) {
        double *o = partial + (size_t)it * 14;
        o[0] = 0.5 * u0;
        o[1] = 0.5 * u1;
#pragma unroll
        for (int k = 0; k < 12; ++k) o[2 + k] = 0.5 * (double)wv[k];
    }
}

// ---------------------------------------------------------------------------
// FP64 kernel (same structure)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * WPB)
k_pair_f64(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
           const int *__restrict__ count, const int2 *__restrict__ items, int n_items,
           const double4 *__restrict__ posd, const int2 *__restrict__ aux, const int *__restrict__ sidx, int sub,
           double *__restrict__ F, double *__restrict__ partial, const PairConstsD pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    unsigned *q = reinterpret_cast<unsigned *>(smem) + warp * QCAP * 32;
    double4 *off = reinterpret_cast<double4 *>(smem + WPB * QCAP * 32 * sizeof(unsigned)) + warp * kMaxNb;
    unsigned char *qc = smem + WPB * QCAP * 32 * sizeof(unsigned) + WPB * kMaxNb * sizeof(double4) + warp * QCAP * 32;
    const int it = blockIdx.x * WPB + warp;
    if (it >= n_items) return;
    const int2 item = items[it];
    if (item.x < 0) return;
    const int gc = item.x;
    const DevSys &d = sys[cell_sys[gc]];
    const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
    const int lc = gc - d.cell0;
    const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
    const double wx = d.w[0], wy = d.w[1], wz = d.w[2];
    const int span = 2 * sub + 1;
    for (int nb = lane; nb < span * span * span; nb += 32)
        off[nb] = make_double4((nb % span - sub) * wx, ((nb / span) % span - sub) * wy,
                               (nb / (span * span) - sub) * wz, 0.0);
    __syncwarp();
    const int i0 = start[gc] + 32 * item.y;
    const int ni = min(32, count[gc] - 32 * item.y);
    const bool vi = lane < ni;
    double4 pi = make_double4(0, 0, 0, 0);
    int2 ai = make_int2(-0x7fffffff, 0);
    if (vi) { pi = posd[i0 + lane]; ai = aux[i0 + lane]; }
    const double rc2 = pc.rc2;
    AccD acc;
    acc.fx = acc.fy = acc.fz = 0.0;
    acc.uc = acc.ul = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.wc[k] = acc.wl[k] = 0.0;
    int head = 0, tail = 0;

    auto eval_one = [&](unsigned j, int code) {
        const double4 pj = posd[j];
        const int tj = aux[j].y;
        const double4 o = off[code];
        pair_eval(pc, (pi.x - o.x) - pj.x, (pi.y - o.y) - pj.y, (pi.z - o.z) - pj.z, pi.w, ai.y, pj.w, tj, acc);
    };

    for (int nb = 0; nb < span * span * span; ++nb) {
        const int ddx = nb % span - sub, ddy = (nb / span) % span - sub, ddz = nb / (span * span) - sub;
        const int g = d.cell0 + wrapi(cx + ddx, n0) + n0 * (wrapi(cy + ddy, n1) + n1 * wrapi(cz + ddz, n2));
        const int j0 = start[g], nj = count[g];
        const int code = nb;
        const double4 o = off[nb];
        const double xi = pi.x - o.x, yi = pi.y - o.y, zi = pi.z - o.z;
        for (int jb = 0; jb < nj; jb += 32) {
            const int je = min(jb + 32, nj);
            for (int j = jb; j < je; ++j) {
                const double4 pj = posd[j0 + j];
                const double dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (vi && r2 < rc2 && aux[j0 + j].x != ai.x) {
                    const int slot = (tail & (QCAP - 1)) * 32 + lane;
                    q[slot] = (unsigned)(j0 + j);
                    qc[slot] = (unsigned char)code;
                    ++tail;
                }
            }
            const int mn = __reduce_min_sync(0xffffffffu, vi ? tail - head : QCAP);
            for (int t = 0; t < mn; ++t) {
                if (vi) {
                    const int slot = (head & (QCAP - 1)) * 32 + lane;
                    ++head;
                    eval_one(q[slot], qc[slot]);
                }
            }
            while (__reduce_max_sync(0xffffffffu, tail - head) > QCAP - 32) {
                if (tail > head) {
                    const int slot = (head & (QCAP - 1)) * 32 + lane;
                    ++head;
                    eval_one(q[slot], qc[slot]);
                }
            }
        }
    }
    while (__any_sync(0xffffffffu, tail > head)) {
        if (tail > head) {
            const int slot = (head & (QCAP - 1)) * 32 + lane;
            ++head;
            eval_one(q[slot], qc[slot]);
        }
    }
    if (vi) {
        const int ia = sidx[i0 + lane];
        F[3 * ia] = acc.fx;
        F[3 * ia + 1] = acc.fy;
        F[3 * ia + 2] = acc.fz;
    }
    const double v[14] = {acc.uc, acc.ul, acc.wc[0], acc.wc[1], acc.wc[2], acc.wc[3], acc.wc[4],
                          acc.wc[5], acc.wl[0], acc.wl[1], acc.wl[2], acc.wl[3], acc.wl[4], acc.wl[5]};
    double red[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) red[k] = warp_sum(v[k]);
    if (lane == 0) {
        double *o = partial + (size_t)it * 14;
#pragma unroll
        for (int k = 0; k < 14; ++k) o[k] = 0.5 * red[k];
    }
}

// Opt the pair kernels into their dynamic shared memory (once per context,
// outside any stream capture).
cudaError_t prepare_pair()
{
    cudaError_t e = cudaFuncSetAttribute(k_pair_f32<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem(1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_f32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem(1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pair_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem(0));
    return e;
}

void launch_pair(const Batch &b, const AtomArrays &a, int precision, const PairConstsF &cf,
                 const PairConstsD &cd, double *partial, cudaStream_t st)
{
    const int blocks = (b.item_cap + WPB - 1) / WPB;
    const size_t sm = pair_smem(precision);
    if (precision == 1) {
        if (cf.M == 10)
            k_pair_f32<10><<<blocks, 32 * WPB, sm, st>>>(b.sys, b.cell_sys, a.start, a.count, a.items, b.item_cap,
                                                        a.pos4, a.qt, a.sidx, b.sub, a.F, partial, cf);
        else
            k_pair_f32<0><<<blocks, 32 * WPB, sm, st>>>(b.sys, b.cell_sys, a.start, a.count, a.items, b.item_cap,
                                                       a.pos4, a.qt, a.sidx, b.sub, a.F, partial, cf);
    } else {
        k_pair_f64<<<blocks, 32 * WPB, sm, st>>>(b.sys, b.cell_sys, a.start, a.count, a.items, b.item_cap, a.posd,
                                                a.aux, a.sidx, b.sub, a.F, partial, cd);
    }
}

}  // namespace rbsog
