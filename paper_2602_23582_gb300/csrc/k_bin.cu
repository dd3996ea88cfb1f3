// k_bin.cu -- cell lists rebuilt every step (the box rescales each step).
//
// Binning convention (an evaluation outside the NPT step matches the oracle's
// definition bit for bit; no FMA in the decision arithmetic; the NPT step's
// atom update takes s = r (1/L) instead): s = r / L, s -= floor(s), s = 0 if s >= 1;
// n = floor(L * sub / r_c) cells per axis; cell = min(floor(s n), n - 1),
// x fastest.  A tilted cell h: s = h^{-1} r (back substitution) and n from
// the perpendicular widths instead of the edges; cell-local coordinates are
// h (s - c / n), and the offset of neighbour cell c + d is h (d / n).  A warp-aggregated counting sort (match_any + one atomicAdd per
// distinct cell in the warp) gives every atom a rank in its cell; an
// exclusive scan gives the cell starts; atoms are scattered to their cell and
// each cell's list is then sorted, so the cell-sorted order (and every sum
// over it) is deterministic.  FP64 build: by original index.  FP32 build:
// along a snake path through the cell -- kc x kc sub-columns in boustrophedon
// order, z up and down in alternate columns, ties by original index -- so
// that every kClus consecutive atoms (a cluster of the pair kernel) lie close
// together; the same pass writes each cluster's bounding box.
//
// Lists with a skin (FP32 build, NPT steps): cells are r_list / sub wide,
// r_list = r_c + skin, and the binning, scan, scatter, cell sort and list
// build run only for systems flagged for a rebuild (DevSys::rebuild); the
// others keep their cell-sorted order and lists, and k_refresh writes their
// atoms' current coordinates relative to the cells of the last build.
#include "internal.h"

namespace rbsog {

__global__ void k_box_prep(DevSys *sys, int S, int sub, double rc)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    DevSys &d = sys[s];
    d.rebuild = 1;                            // an evaluation outside the NPT step: fresh lists
    const int minc = 2 * sub + 1;
    if (live_n(d) == 0) {                     // empty slot: a valid grid, no checks
        for (int a = 0; a < 3; ++a) { d.ncell[a] = minc; d.w[a] = 1.0; }
        return;
    }
    bool bad = false;
    for (int a = 0; a < 3; ++a) {
        // a box that is too small, not finite or beyond the allocated grid is
        // flagged; the grid stays within [2 sub + 1, ncap] so that every
        // neighbour-cell index remains valid while the step is discarded.
        // A tilted cell is cut along its perpendicular widths, so that the
        // neighbour cells within sub steps hold every pair within r_c.
        const double span = d.tri ? perp_width(d.L, d.tilt, a) : d.L[a];
        const int n = axis_cells(span, sub, rc, d.ncap[a], &bad);
        d.ncell[a] = n;
        d.w[a] = d.L[a] / n;
    }
    d.tw[0] = d.tilt[0] / d.ncell[1];
    d.tw[1] = d.tilt[1] / d.ncell[2];
    d.tw[2] = d.tilt[2] / d.ncell[2];
    if (bad) d.flags |= FLAG_BOX;
    d.V = d.L[0] * d.L[1] * d.L[2];
}

__global__ void k_clear_flags(DevSys *sys, int S)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) sys[s].flags = 0;
}

void launch_clear_flags(const Batch &b, cudaStream_t st)
{
    k_clear_flags<<<(b.S + 127) / 128, 128, 0, st>>>(b.sys, b.S);
}

void launch_box_prep(const Batch &b, cudaStream_t st)
{
    k_box_prep<<<(b.S + 127) / 128, 128, 0, st>>>(b.sys, b.S, b.sub, b.rlist);
}

__global__ void k_invalidate_lists(DevSys *sys, int S)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) sys[s].list_valid = 0;
}

void launch_invalidate_lists(const Batch &b, cudaStream_t st)
{
    k_invalidate_lists<<<(b.S + 127) / 128, 128, 0, st>>>(b.sys, b.S);
}

__global__ void k_bin(const DevSys *__restrict__ sys, const int *__restrict__ atom_sys,
                      const double *__restrict__ r, const double *__restrict__ q,
                      const int *__restrict__ mol, int N, int *__restrict__ cell,
                      int *__restrict__ rank, int *__restrict__ count, float4 *__restrict__ locf,
                      double4 *__restrict__ locd, uint4 *__restrict__ su, double *__restrict__ xref,
                      int precision)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool live = false;
    if (i < N) {
        const DevSys &ds = sys[atom_sys[i]];
        if (ds.rebuild) {                     // else the atom keeps the cell of the last build
            live = i - ds.atom0 < live_n(ds); // slots hold up to their capacity
            if (!live) cell[i] = -1;
        }
    }
    const unsigned act = __ballot_sync(0xffffffffu, live);
    if (!live) return;
    const DevSys &d = sys[atom_sys[i]];
    const double x[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
    bin_atom(d, i, x, q[i], mol[i], act, cell, rank, count, locf, locd, su, precision);
    xref[3 * i] = x[0];
    xref[3 * i + 1] = x[1];
    xref[3 * i + 2] = x[2];
}

void launch_bin(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st, bool zero_counts)
{
    if (zero_counts) cudaMemsetAsync(a.count, 0, sizeof(int) * b.C, st);
    k_bin<<<(b.N + 255) / 256, 256, 0, st>>>(b.sys, b.atom_sys, a.r, a.q, a.mol, b.N, a.cell, a.rank,
                                             a.count, a.locf, a.locd, a.su, a.xref, precision);
}

// Atoms of systems that keep their lists: cell-local coordinates relative to
// the cell of the last build (the image nearest that cell; the cell widths
// follow the box) and fixed-point fractional coordinates, as bin_atom forms
// them.  One thread per cell-sorted slot.
__global__ void k_refresh(const DevSys *__restrict__ sys, const int *__restrict__ atom_sys,
                          const double *__restrict__ r, const double *__restrict__ q, const int *__restrict__ mol,
                          const int *__restrict__ sidx, const int *__restrict__ cell, const int *__restrict__ start,
                          const int2 *__restrict__ ccl, int N, float4 *__restrict__ pos4, uint4 *__restrict__ su)
{
    const int ks = blockIdx.x * blockDim.x + threadIdx.x;
    if (ks >= N) return;
    const DevSys &d = sys[atom_sys[ks]];      // sorted slots keep their system's range
    if (d.rebuild || ks - d.atom0 >= live_n(d)) return;
    const int i = sidx[ks];
    const int lc = cell[i] - d.cell0;
    const int k[3] = {lc % d.ncell[0], (lc / d.ncell[0]) % d.ncell[1], lc / (d.ncell[0] * d.ncell[1])};
    double sf[3], xl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double L = d.L[a];
        double s = __ddiv_rn(r[3 * i + a], L);
        s = __dsub_rn(s, floor(s));
        if (s >= 1.0) s = 0.0;
        sf[a] = s;
        double x = s * L - k[a] * d.w[a];
        x -= L * rint(x / L);
        xl[a] = x;
    }
    // cluster slot of the atom: the cell's clusters start at item ccl.x
    const int g = cell[i], kc = ks - start[g];
    pos4[kClus * (ccl[g].x + kc / kClus) + kc % kClus] =
        make_float4((float)xl[0], (float)xl[1], (float)xl[2], __int_as_float(mol[i]));
    su[i] = make_uint4(__double2uint_rz(sf[0] * 4294967296.0), __double2uint_rz(sf[1] * 4294967296.0),
                       __double2uint_rz(sf[2] * 4294967296.0), __float_as_uint((float)q[i]));
}

void launch_refresh(const Batch &b, const AtomArrays &a, cudaStream_t st)
{
    k_refresh<<<(b.N + 255) / 256, 256, 0, st>>>(b.sys, b.atom_sys, a.r, a.q, a.mol, a.sidx, a.cell, a.start,
                                                 a.ccl, b.N, a.pos4, a.su);
}

// Per-system exclusive scan of the cell counts (one block per system): the
// atoms of system s occupy [atom0, atom0 + n) of the sorted arrays.  The same
// pass lists the pair kernel's work items of the system in [item0, item0 +
// nitems) and marks the rest of its item range unused.  An item is (cell g,
// k): the k-th group of gsize atoms of cell g (FP64: 32-atom groups; FP32:
// clusters of kClus atoms, and ccl[g] = (first item of cell g, its items)).
// Each thread lists the cells of its own range, in order.
__device__ __forceinline__ int scan_items(const int *__restrict__ count, int C0, int c0, int c1, int gsize,
                                          int2 *__restrict__ items, int2 *__restrict__ ccl, int rg, bool write)
{
    int ni = 0;
    for (int c = c0; c < c1; ++c) {
        const int v = min(count[C0 + c], kCellCap);
        const int ng = (v + gsize - 1) / gsize;
        if (write) {
            if (ccl) ccl[C0 + c] = make_int2(rg + ni, ng);
            for (int g = 0; g < ng; ++g) items[rg + ni + g] = make_int2(C0 + c, g);
        }
        ni += ng;
    }
    return ni;
}

__global__ void __launch_bounds__(1024)
k_scan(const int *__restrict__ count, int *__restrict__ start, int2 *__restrict__ items, int2 *__restrict__ ccl,
       DevSys *sys, int gsize)
{
    __shared__ int ta[1024], tg[1024];
    DevSys &d = sys[blockIdx.x];
    if (!d.rebuild) return;                  // block-uniform: the system keeps its lists
    const int t = threadIdx.x, T = blockDim.x;
    const int C0 = d.cell0, nc = d.ncell_cap_total;
    const int per = (nc + T - 1) / T;
    const int c0 = min(nc, t * per), c1 = min(nc, c0 + per);
    int sa = 0;
    for (int c = c0; c < c1; ++c) {
        const int v = count[C0 + c];
        if (v > kCellCap) atomicOr(&d.flags, (int)FLAG_OVERFLOW);
        sa += v;
    }
    const int sg = scan_items(count, C0, c0, c1, gsize, items, ccl, 0, false);
    ta[t] = sa;
    tg[t] = sg;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        int va = (t >= o) ? ta[t - o] : 0, vg = (t >= o) ? tg[t - o] : 0;
        __syncthreads();
        ta[t] += va;
        tg[t] += vg;
        __syncthreads();
    }
    int ra = d.atom0 + ta[t] - sa;
    const int rg = d.item0 + tg[t] - sg;
    for (int c = c0; c < c1; ++c) {
        start[C0 + c] = ra;
        ra += count[C0 + c];
    }
    scan_items(count, C0, c0, c1, gsize, items, ccl, rg, true);
    const int total = tg[T - 1];
    if (t == T - 1) {
        d.nitems = total;
        d.Lref[0] = d.L[0]; d.Lref[1] = d.L[1]; d.Lref[2] = d.L[2];
        d.list_valid = 1;
        ++d.list_builds;
    }
    for (int k = total + t; k < d.item_cap; k += T) items[d.item0 + k] = make_int2(-1, -1);
}

void launch_scan(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st)
{
    k_scan<<<b.S, 1024, 0, st>>>(a.count, a.start, a.items, precision == 1 ? a.ccl : nullptr, b.sys,
                                 precision == 1 ? kClus : 32);
}

__global__ void k_scatter(const DevSys *__restrict__ sys, const int *__restrict__ atom_sys,
                          const int *__restrict__ cell, const int *__restrict__ rank,
                          const int *__restrict__ start, int *__restrict__ sidx, int N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || !sys[atom_sys[i]].rebuild || cell[i] < 0) return;
    sidx[start[cell[i]] + rank[i]] = i;
}

// One block per cell: bitonic sort of the cell's atom list by a 64-bit key
// (kSortThreads threads, each stage one compare-exchange per thread for a
// cell of up to 2 kSortThreads atoms), then gather the cell-sorted copies used
// by the pair kernel.  FP64: key = original index.  FP32: key = (sub-column
// along the snake path) << 48 | (z position along the column's direction,
// 16 bits) << 32 | original index; then the bounding box of each cluster of
// kClus consecutive atoms (centre, half extent; cell-local coordinates).
constexpr int kSortThreads = 128;

__device__ __forceinline__ unsigned long long snake_key(float4 l, const DevSys &d, int i)
{
    const int kc = d.kc;
    const float fx = l.x / (float)d.w[0], fy = l.y / (float)d.w[1], fz = l.z / (float)d.w[2];
    const int sx = min(kc - 1, max(0, (int)(fx * (float)kc)));
    const int sy = min(kc - 1, max(0, (int)(fy * (float)kc)));
    const int col = sy * kc + ((sy & 1) ? kc - 1 - sx : sx);
    unsigned zq = (unsigned)(fminf(fmaxf(fz, 0.f), 1.f) * 65535.f);
    if (col & 1) zq = 65535u - zq;
    return ((unsigned long long)col << 48) | ((unsigned long long)zq << 32) | (unsigned)i;
}

__global__ void __launch_bounds__(kSortThreads)
k_cell_sort(const DevSys *__restrict__ sys, const int *__restrict__ cell_sys, const int *__restrict__ start,
            const int *__restrict__ count, int C, int *__restrict__ sidx, int *__restrict__ rank,
            const float4 *__restrict__ locf, const double4 *__restrict__ locd, const double *__restrict__ q,
            const int *__restrict__ type, const int *__restrict__ mol, float4 *__restrict__ pos4,
            float2 *__restrict__ qt, double4 *__restrict__ posd, float4 *__restrict__ posf,
            int2 *__restrict__ aux, const int2 *__restrict__ ccl, float4 *__restrict__ cbox, int precision)
{
    __shared__ unsigned long long s[kCellCap];
    const int c = blockIdx.x, t0 = threadIdx.x;
    const int base = start[c];
    const int n = min(count[c], kCellCap);
    if (n == 0) return;                                // block-uniform (and systems that keep their lists)
    const DevSys &d = sys[cell_sys[c]];
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int k = t0; k < p2; k += kSortThreads) {
        unsigned long long key = ~0ull;
        if (k < n) {
            const int i = sidx[base + k];
            key = precision == 1 ? snake_key(locf[i], d, i) : (unsigned long long)(unsigned)i;
        }
        s[k] = key;
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = t0; t < p2 / 2; t += kSortThreads) {
                int lo = 2 * j * (t / j) + (t % j);
                int hi = lo + j;
                bool up = (lo & k) == 0;
                const unsigned long long x = s[lo], y = s[hi];
                if ((x > y) == up) { s[lo] = y; s[hi] = x; }
            }
            __syncthreads();
        }
    }
    int2 cc = make_int2(0, 0);
    if (precision == 1) cc = ccl[c];
    for (int k = t0; k < n; k += kSortThreads) {
        const int i = (int)(unsigned)(s[k] & 0xffffffffull);
        sidx[base + k] = i;
        rank[i] = base + k;          // from here on: cell-sorted position of atom i
        if (precision == 1) {
            // cluster slot k % kClus of the cell's cluster k / kClus
            const int slot = kClus * (cc.x + k / kClus) + k % kClus;
            pos4[slot] = locf[i];
            qt[slot] = make_float2((float)q[i], __int_as_float(type[i]));
        } else {
            const double4 l = locd[i];
            posd[base + k] = l;
            posf[base + k] = make_float4((float)l.x, (float)l.y, (float)l.z, __int_as_float(mol[i]));
            aux[base + k] = make_int2(mol[i], type[i]);
        }
    }
    if (precision != 1) return;
    // the unused slots of the last cluster: a far-away atom of no molecule
    for (int k = n + t0; k < kClus * cc.y; k += kSortThreads) {
        const int slot = kClus * (cc.x + k / kClus) + k % kClus;
        pos4[slot] = make_float4(1e15f, 1e15f, 1e15f, __int_as_float(-2));
        qt[slot] = make_float2(0.f, __int_as_float(0));
    }
    for (int k = t0; k < cc.y; k += kSortThreads) {
        const int a0 = kClus * k, na = min(kClus, n - a0);
        float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
        for (int j = 0; j < na; ++j) {
            const float4 v = locf[(int)(unsigned)(s[a0 + j] & 0xffffffffull)];
            lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
            hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
        }
        cbox[2 * (cc.x + k)] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]),
                                           __int_as_float(base + a0));
        cbox[2 * (cc.x + k) + 1] = make_float4(0.5f * (hi[0] - lo[0]), 0.5f * (hi[1] - lo[1]),
                                               0.5f * (hi[2] - lo[2]), __int_as_float(na));
    }
}

// Bounding boxes of the clusters of systems that keep their lists (their
// atoms' coordinates were refreshed in the cells of the last build); one
// thread per work item.
__global__ void k_cluster_box(const DevSys *__restrict__ sys, const int *__restrict__ item_sys, int item_cap,
                              const int2 *__restrict__ items, const float4 *__restrict__ pos4,
                              float4 *__restrict__ cbox)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= item_cap) return;
    const DevSys &d = sys[item_sys[it]];
    if (d.rebuild || live_n(d) == 0 || it - d.item0 >= d.nitems || items[it].x < 0) return;
    const float4 b0 = cbox[2 * it], b1 = cbox[2 * it + 1];
    const int na = __float_as_int(b1.w);
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    for (int j = 0; j < na; ++j) {
        const float4 v = pos4[kClus * it + j];
        lo[0] = fminf(lo[0], v.x); lo[1] = fminf(lo[1], v.y); lo[2] = fminf(lo[2], v.z);
        hi[0] = fmaxf(hi[0], v.x); hi[1] = fmaxf(hi[1], v.y); hi[2] = fmaxf(hi[2], v.z);
    }
    cbox[2 * it] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]), b0.w);
    cbox[2 * it + 1] = make_float4(0.5f * (hi[0] - lo[0]), 0.5f * (hi[1] - lo[1]), 0.5f * (hi[2] - lo[2]), b1.w);
}

void launch_cluster_box(const Batch &b, const AtomArrays &a, cudaStream_t st)
{
    k_cluster_box<<<(b.item_cap + 255) / 256, 256, 0, st>>>(b.sys, b.item_sys, b.item_cap, a.items, a.pos4, a.cbox);
}

void launch_scatter_sort(const Batch &b, const AtomArrays &a, int precision, cudaStream_t st)
{
    k_scatter<<<(b.N + 127) / 128, 128, 0, st>>>(b.sys, b.atom_sys, a.cell, a.rank, a.start, a.sidx, b.N);
    k_cell_sort<<<b.C, kSortThreads, 0, st>>>(b.sys, b.cell_sys, a.start, a.count, b.C, a.sidx, a.rank, a.locf,
                                              a.locd, a.q, a.type, a.mol, a.pos4, a.qt, a.posd, a.posf, a.aux,
                                              a.ccl,
                                              a.cbox, precision);
}

}  // namespace rbsog
