// k_pair.cu -- SOG short-range pair forces, energy and virial over cell lists
// (paper sec. 2.2 and 3.1; eqs. force_SOG, U_short, P_short) plus a 12-6
// Lennard-Jones term cut (unshifted) at r_c.
//
// Per pair with r < r_c and different molecule ids:
//   f   = ke q_i q_j (1/r^3 - sum_{l<M} w~_l e^{-r^2/s~_l^2}) r_vec   (kernel N~)
//   U  += ke q_i q_j (1/r   - sum_{l<ME} w_l e^{-r^2/s_l^2})          (kernel N)
//   W  += f (x) r_vec  (eq. P_short: P^N = W / V)
// Full pairs: every atom's block sums all its neighbours (no atomics, so the
// result does not depend on scheduling); energies and virials take half.
//
// One block per home cell.  Each warp owns 32 i-atoms (one per lane, in
// registers).  For each row of neighbour cells (fixed dy, dz; dx in
// [-sub, sub]) the block stages the row's atoms into shared memory with the
// periodic offset already added (coordinates are cell-local, so FP32 keeps
// ~1e-6 A).  Lanes test candidates (distance and molecule id only) and push
// the hits into per-lane queues; the warp evaluates queued hits in rounds in
// which every lane has one, so the 11-transcendental SOG kernel never runs
// with idle lanes except when queues are drained at the end of a tile.
#include "internal.h"

namespace rbsog {

namespace {

constexpr int QCAP = 64;   // per-lane hit queue (power of two); pending <= 32 before a batch
constexpr int JT = 512;    // atoms per staged tile

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct AccF {
    float fx, fy, fz;
    float uc, ul;
    float wc[6], wl[6];
};

template <int NG>
__device__ __forceinline__ void pair_eval_f(const PairConstsF &pc, float xi, float yi, float zi,
                                            float qi, int ti, float4 pj, float2 qj, AccF &acc)
{
    const float dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
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
    acc.uc += ec;
    acc.ul += el;
    const float cx = fc * dx, cy = fc * dy, lx = fl * dx, ly = fl * dy;
    acc.wc[0] = fmaf(cx, dx, acc.wc[0]); acc.wc[1] = fmaf(cy, dy, acc.wc[1]);
    acc.wc[2] = fmaf(fc * dz, dz, acc.wc[2]); acc.wc[3] = fmaf(cx, dy, acc.wc[3]);
    acc.wc[4] = fmaf(cx, dz, acc.wc[4]); acc.wc[5] = fmaf(cy, dz, acc.wc[5]);
    acc.wl[0] = fmaf(lx, dx, acc.wl[0]); acc.wl[1] = fmaf(ly, dy, acc.wl[1]);
    acc.wl[2] = fmaf(fl * dz, dz, acc.wl[2]); acc.wl[3] = fmaf(lx, dy, acc.wl[3]);
    acc.wl[4] = fmaf(lx, dz, acc.wl[4]); acc.wl[5] = fmaf(ly, dz, acc.wl[5]);
}

struct AccD {
    double fx, fy, fz;
    double uc, ul;
    double wc[6], wl[6];
};

__device__ __forceinline__ void pair_eval_d(const PairConstsD &pc, double xi, double yi, double zi,
                                            double qi, int ti, double4 pj, int tj, AccD &acc)
{
    const double dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
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
    const double qq = pc.ke * qi * pj.w;
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

// Row of neighbour cells: up to 5 cells (sub <= 2).
struct RowInfo {
    int start[5], count[5], cum[6];
    float offx[5];
    double offxd[5];
};

__device__ __forceinline__ int find_cell(const RowInfo &ri, int ncr, int k)
{
    int c = 0;
#pragma unroll
    for (int t = 1; t < 5; ++t)
        if (t < ncr && k >= ri.cum[t]) c = t;
    return c;
}

}  // namespace

// ---------------------------------------------------------------------------
// FP32 kernel
// ---------------------------------------------------------------------------
template <int NG>
__global__ void k_pair_f32(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys,
                           const int *__restrict__ start, const float4 *__restrict__ pos4,
                           const float2 *__restrict__ qt, const int *__restrict__ sidx, int sub,
                           double *__restrict__ F, double *__restrict__ partial, const PairConstsF pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nw = blockDim.x >> 5;
    float4 *Jp = reinterpret_cast<float4 *>(smem);
    float2 *Jq = reinterpret_cast<float2 *>(Jp + JT);
    unsigned *queue = reinterpret_cast<unsigned *>(Jq + JT);     // [nw][QCAP][32]
    __shared__ RowInfo ri;
    __shared__ double grp[14][kCellCap / 32];

    const int gc = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const DevSys &d = sys[cell_sys[gc]];
    const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
    const int lc = gc - d.cell0;
    AccF acc;
    int ngroups = 0;

    if (lc < n0 * n1 * n2) {
        const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
        const int i0 = start[gc], ni = start[gc + 1] - i0;
        const float wx = (float)d.w[0], wy = (float)d.w[1], wz = (float)d.w[2];
        const int ncr = 2 * sub + 1;
        unsigned *q = queue + warp * QCAP * 32;
        const int rounds = (ni + 32 * nw - 1) / (32 * nw);
        ngroups = (min(ni, kCellCap) + 31) / 32;
        for (int rd = 0; rd < rounds; ++rd) {
            const int il = rd * 32 * nw + warp * 32 + lane;
            const bool vi = il < ni;
            acc.uc = acc.ul = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc.wc[k] = acc.wl[k] = 0.f;
            float4 pi = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            float2 pq = make_float2(0.f, 0.f);
            if (vi) { pi = pos4[i0 + il]; pq = qt[i0 + il]; }
            const int moli = vi ? __float_as_int(pi.w) : -0x7fffffff;
            const int ti = __float_as_int(pq.y);
            acc.fx = acc.fy = acc.fz = 0.f;
            for (int dz = -sub; dz <= sub; ++dz) {
                for (int dy = -sub; dy <= sub; ++dy) {
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        int yy = cy + dy, zz = cz + dz;
                        yy += (yy < 0) ? n1 : ((yy >= n1) ? -n1 : 0);
                        zz += (zz < 0) ? n2 : ((zz >= n2) ? -n2 : 0);
                        ri.cum[0] = 0;
                        for (int t = 0; t < ncr; ++t) {
                            int xx = cx + t - sub;
                            xx += (xx < 0) ? n0 : ((xx >= n0) ? -n0 : 0);
                            int g = d.cell0 + xx + n0 * (yy + n1 * zz);
                            ri.start[t] = start[g];
                            ri.count[t] = start[g + 1] - start[g];
                            ri.cum[t + 1] = ri.cum[t] + ri.count[t];
                            ri.offx[t] = (float)((t - sub) * d.w[0]);
                        }
                    }
                    __syncthreads();
                    const int total = ri.cum[ncr];
                    const float oy = dy * wy, oz = dz * wz;
                    for (int base = 0; base < total; base += JT) {
                        const int nj = min(JT, total - base);
                        __syncthreads();
                        for (int k = threadIdx.x; k < nj; k += blockDim.x) {
                            int kk = base + k;
                            int c = find_cell(ri, ncr, kk);
                            int src = ri.start[c] + (kk - ri.cum[c]);
                            float4 p = pos4[src];
                            p.x += ri.offx[c];
                            p.y += oy;
                            p.z += oz;
                            Jp[k] = p;
                            Jq[k] = qt[src];
                        }
                        __syncthreads();
                        // candidates + queued evaluation (per warp)
                        int head = 0, tail = 0;
                        if (!__any_sync(0xffffffffu, vi)) continue;
                        for (int jb = 0; jb < nj; jb += 32) {
                            const int je = min(jb + 32, nj);
                            for (int j = jb; j < je; ++j) {
                                const float4 pj = Jp[j];
                                const float dx = pi.x - pj.x, dy2 = pi.y - pj.y, dz2 = pi.z - pj.z;
                                const float r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
                                if (vi && r2 < pc.rc2 && __float_as_int(pj.w) != moli) {
                                    q[(tail & (QCAP - 1)) * 32 + lane] = (unsigned)j;
                                    ++tail;
                                }
                            }
                            // rounds in which every lane holding an atom has a hit queued;
                            // lanes without an atom have nothing queued and sit them out
                            int pend = tail - head;
                            int mn = __reduce_min_sync(0xffffffffu, vi ? pend : QCAP);
                            for (int t = 0; t < mn; ++t) {
                                if (vi) {
                                    unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                    ++head;
                                    pair_eval_f<NG>(pc, pi.x, pi.y, pi.z, pq.x, ti, Jp[j], Jq[j], acc);
                                }
                            }
                            while (__reduce_max_sync(0xffffffffu, tail - head) > QCAP - 32) {
                                if (tail > head) {
                                    unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                    ++head;
                                    pair_eval_f<NG>(pc, pi.x, pi.y, pi.z, pq.x, ti, Jp[j], Jq[j], acc);
                                }
                            }
                        }
                        while (__any_sync(0xffffffffu, tail > head)) {
                            if (tail > head) {
                                unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                ++head;
                                pair_eval_f<NG>(pc, pi.x, pi.y, pi.z, pq.x, ti, Jp[j], Jq[j], acc);
                            }
                        }
                    }
                }
            }
            if (vi) {
                const int ia = sidx[i0 + il];
                F[3 * ia] = acc.fx;
                F[3 * ia + 1] = acc.fy;
                F[3 * ia + 2] = acc.fz;
            }
            // per 32-atom group: FP32 warp sum, kept per group index so that the
            // cell total does not depend on the warps per block
            const int g = rd * nw + warp;
            const float v[14] = {acc.uc, acc.ul, acc.wc[0], acc.wc[1], acc.wc[2], acc.wc[3], acc.wc[4],
                                 acc.wc[5], acc.wl[0], acc.wl[1], acc.wl[2], acc.wl[3], acc.wl[4], acc.wl[5]};
#pragma unroll
            for (int k = 0; k < 14; ++k) {
                float x = warp_sumf(v[k]);
                if (lane == 0 && g < ngroups) grp[k][g] = (double)x;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 14) {
        double s = 0.0;
        for (int g = 0; g < ngroups; ++g) s += grp[threadIdx.x][g];
        partial[(size_t)gc * 14 + threadIdx.x] = 0.5 * s;
    }
}

// ---------------------------------------------------------------------------
// FP64 kernel (same structure)
// ---------------------------------------------------------------------------
__global__ void k_pair_f64(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys,
                           const int *__restrict__ start, const double4 *__restrict__ posd,
                           const int2 *__restrict__ aux, const int *__restrict__ sidx, int sub,
                           double *__restrict__ F, double *__restrict__ partial, const PairConstsD pc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nw = blockDim.x >> 5;
    double4 *Jp = reinterpret_cast<double4 *>(smem);
    int2 *Ja = reinterpret_cast<int2 *>(Jp + JT);
    unsigned *queue = reinterpret_cast<unsigned *>(Ja + JT);
    __shared__ RowInfo ri;
    __shared__ double grp[14][kCellCap / 32];

    const int gc = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const DevSys &d = sys[cell_sys[gc]];
    const int n0 = d.ncell[0], n1 = d.ncell[1], n2 = d.ncell[2];
    const int lc = gc - d.cell0;
    AccD acc;
    int ngroups = 0;

    if (lc < n0 * n1 * n2) {
        const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
        const int i0 = start[gc], ni = start[gc + 1] - i0;
        const int ncr = 2 * sub + 1;
        unsigned *q = queue + warp * QCAP * 32;
        const int rounds = (ni + 32 * nw - 1) / (32 * nw);
        ngroups = (min(ni, kCellCap) + 31) / 32;
        for (int rd = 0; rd < rounds; ++rd) {
            const int il = rd * 32 * nw + warp * 32 + lane;
            const bool vi = il < ni;
            acc.uc = acc.ul = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc.wc[k] = acc.wl[k] = 0.0;
            double4 pi = make_double4(0, 0, 0, 0);
            int2 ai = make_int2(-0x7fffffff, 0);
            if (vi) { pi = posd[i0 + il]; ai = aux[i0 + il]; }
            acc.fx = acc.fy = acc.fz = 0.0;
            for (int dz = -sub; dz <= sub; ++dz) {
                for (int dy = -sub; dy <= sub; ++dy) {
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        int yy = cy + dy, zz = cz + dz;
                        yy += (yy < 0) ? n1 : ((yy >= n1) ? -n1 : 0);
                        zz += (zz < 0) ? n2 : ((zz >= n2) ? -n2 : 0);
                        ri.cum[0] = 0;
                        for (int t = 0; t < ncr; ++t) {
                            int xx = cx + t - sub;
                            xx += (xx < 0) ? n0 : ((xx >= n0) ? -n0 : 0);
                            int g = d.cell0 + xx + n0 * (yy + n1 * zz);
                            ri.start[t] = start[g];
                            ri.count[t] = start[g + 1] - start[g];
                            ri.cum[t + 1] = ri.cum[t] + ri.count[t];
                            ri.offxd[t] = (t - sub) * d.w[0];
                        }
                    }
                    __syncthreads();
                    const int total = ri.cum[ncr];
                    const double oy = dy * d.w[1], oz = dz * d.w[2];
                    for (int base = 0; base < total; base += JT) {
                        const int nj = min(JT, total - base);
                        __syncthreads();
                        for (int k = threadIdx.x; k < nj; k += blockDim.x) {
                            int kk = base + k;
                            int c = find_cell(ri, ncr, kk);
                            int src = ri.start[c] + (kk - ri.cum[c]);
                            double4 p = posd[src];
                            p.x += ri.offxd[c];
                            p.y += oy;
                            p.z += oz;
                            Jp[k] = p;
                            Ja[k] = aux[src];
                        }
                        __syncthreads();
                        int head = 0, tail = 0;
                        if (!__any_sync(0xffffffffu, vi)) continue;
                        for (int jb = 0; jb < nj; jb += 32) {
                            const int je = min(jb + 32, nj);
                            for (int j = jb; j < je; ++j) {
                                const double4 pj = Jp[j];
                                const double dx = pi.x - pj.x, dy2 = pi.y - pj.y, dz2 = pi.z - pj.z;
                                const double r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
                                if (vi && r2 < pc.rc2 && Ja[j].x != ai.x) {
                                    q[(tail & (QCAP - 1)) * 32 + lane] = (unsigned)j;
                                    ++tail;
                                }
                            }
                            int pend = tail - head;
                            int mn = __reduce_min_sync(0xffffffffu, vi ? pend : QCAP);
                            for (int t = 0; t < mn; ++t) {
                                if (vi) {
                                    unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                    ++head;
                                    pair_eval_d(pc, pi.x, pi.y, pi.z, pi.w, ai.y, Jp[j], Ja[j].y, acc);
                                }
                            }
                            while (__reduce_max_sync(0xffffffffu, tail - head) > QCAP - 32) {
                                if (tail > head) {
                                    unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                    ++head;
                                    pair_eval_d(pc, pi.x, pi.y, pi.z, pi.w, ai.y, Jp[j], Ja[j].y, acc);
                                }
                            }
                        }
                        while (__any_sync(0xffffffffu, tail > head)) {
                            if (tail > head) {
                                unsigned j = q[(head & (QCAP - 1)) * 32 + lane];
                                ++head;
                                pair_eval_d(pc, pi.x, pi.y, pi.z, pi.w, ai.y, Jp[j], Ja[j].y, acc);
                            }
                        }
                    }
                }
            }
            if (vi) {
                const int ia = sidx[i0 + il];
                F[3 * ia] = acc.fx;
                F[3 * ia + 1] = acc.fy;
                F[3 * ia + 2] = acc.fz;
            }
            const int g = rd * nw + warp;
            const double v[14] = {acc.uc, acc.ul, acc.wc[0], acc.wc[1], acc.wc[2], acc.wc[3], acc.wc[4],
                                  acc.wc[5], acc.wl[0], acc.wl[1], acc.wl[2], acc.wl[3], acc.wl[4], acc.wl[5]};
#pragma unroll
            for (int k = 0; k < 14; ++k) {
                double x = warp_sum(v[k]);
                if (lane == 0 && g < ngroups) grp[k][g] = x;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 14) {
        double s = 0.0;
        for (int g = 0; g < ngroups; ++g) s += grp[threadIdx.x][g];
        partial[(size_t)gc * 14 + threadIdx.x] = 0.5 * s;
    }
}

size_t pair_smem_bytes(int precision, int nw)
{
    size_t tile = precision == 1 ? (size_t)JT * (sizeof(float4) + sizeof(float2))
                                 : (size_t)JT * (sizeof(double4) + sizeof(int2));
    return tile + (size_t)nw * QCAP * 32 * sizeof(unsigned);
}

// Opt the pair kernels into the dynamic shared memory they need (called once
// per context, outside any stream capture).
cudaError_t prepare_pair(int precision, int nw)
{
    const int sm = (int)pair_smem_bytes(precision, nw);
    cudaError_t e;
    if (precision == 1) {
        e = cudaFuncSetAttribute(k_pair_f32<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_pair_f32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    } else {
        e = cudaFuncSetAttribute(k_pair_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    return e;
}

void launch_pair(const Batch &b, const AtomArrays &a, int precision, const PairConstsF &cf,
                 const PairConstsD &cd, double *partial, int nw, cudaStream_t st)
{
    const size_t sm = pair_smem_bytes(precision, nw);
    if (precision == 1) {
        if (cf.M == 10)
            k_pair_f32<10><<<b.C, 32 * nw, sm, st>>>(b.sys, b.cell_sys, a.start, a.pos4, a.qt, a.sidx,
                                                      b.sub, a.F, partial, cf);
        else
            k_pair_f32<0><<<b.C, 32 * nw, sm, st>>>(b.sys, b.cell_sys, a.start, a.pos4, a.qt, a.sidx,
                                                     b.sub, a.F, partial, cf);
    } else {
        k_pair_f64<<<b.C, 32 * nw, sm, st>>>(b.sys, b.cell_sys, a.start, a.posd, a.aux, a.sidx, b.sub,
                                             a.F, partial, cd);
    }
}

}  // namespace rbsog
