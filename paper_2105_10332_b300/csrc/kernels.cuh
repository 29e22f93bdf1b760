// kernels.cuh -- swept-rule phase kernels and the Standard step kernel.
//
// Geometry (Sec. 3.3; levels are RK stages, n the radius of one stage, b the
// block edge, d the levels one phase advances, 2 <= d <= b/(2n) - 1 (Eq. 1),
// d even).  Every kernel below gives a b x b window of the periodic grid to
// one CTA, or to a thread-block cluster of C CTAs, and takes one shape
// through its levels inside shared memory:
//
//   Up-Pyramid   window = block of the grid (offset o = 0 or b/2 in x and y)
//                level base+s covers [sn, b-sn)^2 of the window
//   X-Bridge     window = block shifted by b/2 in x (the seam in its middle)
//                level base+s covers [b/2-sn, b/2+sn) x [sn, b-sn)
//   Y-Bridge     the same with x and y exchanged
//   Octahedron   window = block shifted by b/2 in x and y (a corner of four
//                blocks in its middle); lower half: [b/2-sn, b/2+sn)^2 at
//                base+s, then an Up-Pyramid on the same window from base+d
//   Down-Pyramid the lower half alone, then the whole window goes to the state
//
// At every level the four kinds partition the plane.  Values that one shape
// hands to another go through a level store in device memory: d+1 full-grid
// slots, level l in slot l mod (d+1).  A shape writes only the values some
// other shape reads -- the 2n-wide frame of every Up-Pyramid level, the two
// 2n-wide bands along a Bridge's seam, and the top level of each shape -- and
// reads and writes only cells of its own window.  The windows of an
// Up-Pyramid or Octahedron launch partition the plane; a block's X- and
// Y-Bridge windows overlap in one quadrant, where the two shapes read some of
// the same values but compute and export disjoint regions.  So no word of a
// slot is written by one cluster and read or written by another within a
// launch.  Within a CTA the full-step levels live in buffer F and the stage
// levels in buffer H; a second stage updates F in place.
//
// Clusters: with C > 1 every CTA of the cluster keeps a full copy of F and H;
// CTA r computes the r-th of C row bands of each level, writes the new values
// into its own buffers and, through distributed shared memory, into every
// peer's, and the cluster barrier at the end of the level makes them visible.
// Each CTA's scratch (pressures, limiter factors, face fluxes) covers only one
// band, so a cluster takes the shape's levels in 1/C of the time per level.
// A CTA may also split its band into `passes` sub-bands taken one after the
// other, which shrinks the scratch again (two CTAs then fit on one SM).
#pragma once

#include <cooperative_groups.h>

#include <cstdint>

#include "numerics.cuh"

namespace sweep {

namespace cg = cooperative_groups;

// Threads per CTA.  An FP64 warp instruction holds its SM sub-partition's
// FP64 pipe for 64 cycles, so a few warps per sub-partition suffice; the
// counts below were measured best per kernel family (Euler 256^2: swept
// kernels 0.723 / 0.735 / 0.748 / 0.734 Gcell-steps/s at 256 / 384 / 512 /
// 768 threads, Standard 0.717 / 0.728 / 0.715 / 0.678; heat 4096^2 swept
// 42.9 / 47.1 / 46.4 at 128 / 256 / 512).  kThreads serves the adjoint's
// per-cell kernels.
constexpr int kThreads = 256;

struct Rect {
    int x0, x1, y0, y1;
    __device__ __forceinline__ int w() const { return x1 > x0 ? x1 - x0 : 0; }
    __device__ __forceinline__ int h() const { return y1 > y0 ? y1 - y0 : 0; }
    __device__ __forceinline__ int area() const { return w() * h(); }
    __device__ __forceinline__ bool empty() const { return x1 <= x0 || y1 <= y0; }
};

__device__ __forceinline__ Rect grow(Rect r, int g) { return {r.x0 - g, r.x1 + g, r.y0 - g, r.y1 + g}; }

// rows [ya, yb) of R: the part of R a CTA of rank r in a cluster of C takes
__device__ __forceinline__ Rect band(Rect R, int r, int C)
{
    const int H = R.h(), q = H / C, m = H % C;
    const int ya = R.y0 + r * q + (r < m ? r : m);
    return {R.x0, R.x1, ya, ya + q + (r < m ? 1 : 0)};
}

__device__ __forceinline__ Rect clip_rows(Rect R, int ya, int yb)
{
    return {R.x0, R.x1, R.y0 > ya ? R.y0 : ya, R.y1 < yb ? R.y1 : yb};
}

// Launch parameters shared by every kernel (passed by value).
struct Params {
    int64_t nx, ny;      // grid
    int b;               // block / window edge
    int d;               // levels per phase
    int tiles_x, tiles_y;
    int std_tile;        // block edge of the Standard kernel
    double c1, c2;       // stage coefficients: heat r/2, r; Euler dt/(2dx), dt/dx
    EulerConst ek;
    int literal;         // limiter orientation as printed
    double *state;       // [ncomp][ny][nx]
    double *ws;          // level store: d+1 slots
    int64_t slot_elems;  // doubles per slot (>= ncomp*nx*ny, padded)
    int passes;          // row bands each CTA takes one after another per level
    // Level history (the adjoint's swept recompute, equation EulerHist):
    // every level l < hist_levels that a kernel computes is also written to
    // the full-grid state array of its level: level 2t (Q^t) at
    // hist_q + t*hist_stride, level 2t+1 (the first stage Q*_t) at
    // hist_qs + t*hist_stride.  Each (cell, level) is computed exactly once
    // in a swept run, so the arrays end up complete.
    double *hist_q, *hist_qs;
    int64_t hist_stride, hist_levels;
    // Device error word (the first 4 bytes of the workspace header), or null:
    // kernels OR in the kErr* bits below; the host reads it with sweep_check.
    unsigned *err;
    int std_tx, std_blocks;  // Standard blocks along x, and in all (nx/std_tile, that x ny/std_tile)
    int check_out;  // this launch writes a run's final state: check it for infinities and NaNs
    int narrow;     // nx * ny < 2^31: cell and block indices of a plane fit in 32 bits
};

// Bits of the device error word.
constexpr unsigned kErrLaunch = 1u;     // a kernel found its launch geometry or shared memory wrong
constexpr unsigned kErrNonFinite = 2u;  // a state value written was an infinity or a NaN

__device__ __forceinline__ void report(const Params &p, unsigned bit)
{
    if (p.err)
        atomicOr(p.err, bit);
}

// bytes of dynamic shared memory this launch was given
__device__ __forceinline__ unsigned dyn_smem_bytes()
{
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// Launch check at kernel entry, compiled into the checked build only
// (SWEEP_CHECKED, libsweep_checked.so): the grid, the block and the shared
// memory the kernel's geometry needs.  The condition is the same for every
// CTA of the launch, so when it fails every CTA returns before any barrier
// (nothing waits on a CTA that left), and CTA 0 reports it.  It costs the
// small latency-bound grids a few per cent per launch (heat 64^2 Standard
// 1.57 -> 1.50 Gcell-steps/s), so the default build leaves it out.
__device__ __forceinline__ bool launch_ok(const Params &p, unsigned grid, unsigned threads,
                                          size_t smem)
{
#ifdef SWEEP_CHECKED
    const bool ok = gridDim.x == grid && blockDim.x == threads && dyn_smem_bytes() >= smem;
    if (!ok && blockIdx.x == 0 && threadIdx.x == 0)
        report(p, kErrLaunch);
    return ok;
#else
    (void)p;
    (void)grid;
    (void)threads;
    (void)smem;
    return true;
#endif
}

// an infinity or a NaN, by the bit pattern (integer pipe only)
__device__ __forceinline__ bool nonfinite(double v)
{
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) ==
           0x7ff0000000000000ull;
}

// ------------------------------------------------------------------ equations

// NC components, stage radius N, threads per CTA of the swept kernels
// (SWEPT_THREADS) and of the Standard kernels (STD_THREADS)
struct Heat {
    static constexpr int NC = 1;
    static constexpr int N = 1;
    static constexpr int SWEPT_THREADS = 256, STD_THREADS = 256;
};
struct Euler {
    static constexpr int NC = 4;
    static constexpr int N = 2;
    static constexpr int SWEPT_THREADS = 512, STD_THREADS = 384;
};
// The same Euler scheme, each computed level also written to the level
// history of Params (the adjoint's swept recompute); a distinct type so that
// the forward kernels carry no trace of it.
struct EulerHist {
    static constexpr int NC = 4;
    static constexpr int N = 2;
    static constexpr int SWEPT_THREADS = 512, STD_THREADS = 384;
};
// Heat with the forward-Euler rule of App. A: every level is a whole step,
// T^{l} = fma(r, t(T^{l-1}), T^{l-1}); nothing reaches back two levels.
struct HeatFE {
    static constexpr int NC = 1;
    static constexpr int N = 1;
    static constexpr int SWEPT_THREADS = 256, STD_THREADS = 256;
};

// Rows of the largest band a CTA computes: regions lie inside [n, wp-n), so
// they are at most wp - 2n rows high, split over C CTAs.
__host__ __device__ constexpr int band_rows(int wp, int n, int C) { return (wp - 2 * n + C - 1) / C; }

// Euler scratch layout (doubles), for window wp and cluster size C:
//   P    (rows+4) x wp      cell pressures, band rows +-2
//   HXP, HXM  rows x wp     half limiter factors along x
//   HYP, HYM  (rows+2) x wp half limiter factors along y, band rows +-1
//   FX   4 x rows x (wp-2n+1)   x-face fluxes
//   FY   4 x (rows+1) x (wp-2n) y-face fluxes
__host__ __device__ constexpr size_t euler_scratch(int wp, int C)
{
    const int r = band_rows(wp, 2, C);  // C: bands per window (cluster size x passes)
    return (size_t)(r + 4) * wp + (size_t)2 * r * wp + (size_t)2 * (r + 2) * wp +
           (size_t)4 * r * (wp - 3) + (size_t)4 * (r + 1) * (wp - 4);
}

// shared-memory bytes of one CTA with window edge wp (a one-component
// equation's odd-level buffer starts one double late, see Block::carve)
template <class EQ>
__host__ __device__ constexpr size_t smem_bytes(int wp, int C)
{
    if (EQ::NC == 1)
        return sizeof(double) * (2 * (size_t)wp * wp + 2);
    return sizeof(double) * ((size_t)8 * wp * wp + euler_scratch(wp, C));
}

// Per-CTA view of shared memory.
//
// Level-store traffic moves in 16-byte pairs of cells (x, x+1) whose global
// x is even (one row of a 2 x 2 block of the store).  For a radius-1
// equation the store's block grid is shifted by one cell on odd levels, so
// the pairs of an odd level start on odd window columns; buffer H then
// starts one double late (kHoff), which puts those pairs on 16-byte
// boundaries of shared memory as well.
template <class EQ, int C>
struct Block {
    static constexpr int kHoff = EQ::N == 1 ? 1 : 0;
    double *buf[2];               // F (even levels), H (odd levels): [NC][wp*wp]
    double *peer[C > 1 ? C : 1];  // Euler/heat: base of each peer's shared buffer (C > 1)
    double *P, *hxp, *hxm, *hyp, *hym, *fx, *fy;  // Euler scratch
    int wp;          // window pitch (edge)
    int plane;       // wp*wp
    int rank;        // rank in the cluster
    int64_t ox, oy;  // global origin of the window

    int bands;       // row bands per level: C x passes

    // Level l lives in slot l mod (d+1) of the level store.  The kernel's
    // first level and its slot are set once (set_levels); every later level
    // of the launch, at most 2d above it, finds its slot by subtraction
    // instead of a 64-bit division per access.
    int64_t lbase;
    int sbase;
    __device__ void set_levels(const Params &p, int64_t base)
    {
        lbase = base;
        sbase = (int)(base % (p.d + 1));
    }
    __device__ __forceinline__ double *slot(const Params &p, int64_t level) const
    {
        const int d1 = p.d + 1;
        int sl = (int)(level - lbase) + sbase;
        if (sl >= d1) sl -= d1;
        if (sl >= d1) sl -= d1;
        return p.ws + (int64_t)sl * p.slot_elems;
    }

    // buffer of a level (F for even levels, H for odd).  A select on the
    // parity, not an index into buf[]: an array indexed at run time would
    // live in local memory, and so would every field of the block.
    __device__ __forceinline__ double *lev(int64_t level) const { return (level & 1) ? buf[1] : buf[0]; }

    __device__ void carve(double *smem, int wp_, int passes = 1)
    {
        bands = C * passes;
        wp = wp_;
        plane = wp * wp;
        buf[0] = smem;
        buf[1] = smem + EQ::NC * plane + kHoff;
        rank = 0;
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            rank = (int)cl.block_rank();
            for (int r = 0; r < C; ++r)
                peer[r] = cl.map_shared_rank(smem, r);
        }
        if constexpr (EQ::NC == 4) {
            const int rows = band_rows(wp, EQ::N, bands);
            double *p = smem + 2 * EQ::NC * plane;
            P = p;
            p += (rows + 4) * wp;
            hxp = p;
            p += rows * wp;
            hxm = p;
            p += rows * wp;
            hyp = p;
            p += (rows + 2) * wp;
            hym = p;
            p += (rows + 2) * wp;
            fx = p;
            p += 4 * rows * (wp - 3);
            fy = p;
        }
    }
    // value v of component c at smem index i of the buffer of `level`: into
    // this CTA's copy and every peer's
    __device__ __forceinline__ void put(int64_t level, int c, int i, double v)
    {
        const int off = (int)(level & 1) * (EQ::NC * plane + kHoff) + c * plane + i;
        buf[0][off] = v;
        if constexpr (C > 1) {
#pragma unroll
            for (int r = 0; r < C; ++r)
                if (r != rank) peer[r][off] = v;
        }
    }
};

template <int C>
__device__ __forceinline__ void level_barrier()
{
    if constexpr (C > 1)
        cg::this_cluster().sync();
    else
        __syncthreads();
}

__device__ __forceinline__ int64_t gidx(const Params &p, int64_t ox, int64_t oy, int x, int y)
{
    if (p.narrow) {  // the same arithmetic in 32 bits
        const int nx = (int)p.nx, ny = (int)p.ny;
        int gx = (int)ox + x, gy = (int)oy + y;
        if (gx < 0) gx += nx;
        if (gx >= nx) gx -= nx;
        if (gy < 0) gy += ny;
        if (gy >= ny) gy -= ny;
        return (int64_t)(gy * nx + gx);
    }
    int64_t gx = ox + x, gy = oy + y;
    // windows start inside [0, n) and extend at most one grid period
    if (gx < 0) gx += p.nx;
    if (gx >= p.nx) gx -= p.nx;
    if (gy < 0) gy += p.ny;
    if (gy >= p.ny) gy -= p.ny;
    return gy * p.nx + gx;
}

// Visit one rectangle R with the CTA's threads in units: the pair of cells
// (x, x+1) when `vec` is set and R starts on a window column x = par (mod 2)
// and is an even number of cells wide (f gets two = true), else one cell.
template <class F>
__device__ __forceinline__ void for_rect_units(Rect R, int par, bool vec, F &&f)
{
    const int w = R.w(), h = R.h();
    if (w == 0 || h == 0)
        return;
    const bool two = vec && ((R.x0 - par) & 1) == 0 && (w & 1) == 0;
    const int wu = two ? w >> 1 : w, step = two ? 2 : 1;
    const int total = wu * h;
    for (int q = threadIdx.x; q < total; q += blockDim.x)
        f(R.x0 + (q % wu) * step, R.y0 + q / wu, two);
}

// Visit O \ I (I inside O or empty) in the units of for_rect_units, the
// parts below I, above I (full width), left of I and right of I packed into
// one index space, so that no lane idles while work is left and the whole
// of O \ I costs one loop (these copies lie on the critical path of small
// shapes, where one loop per part would cost four loops' latency).
template <class F>
__device__ __forceinline__ void for_units(Rect O, Rect I, int par, bool vec, F &&f)
{
    if (O.empty())
        return;
    if (I.empty()) {
        for_rect_units(O, par, vec, f);
        return;
    }
    const Rect a = {O.x0, O.x1, O.y0, I.y0}, b = {O.x0, O.x1, I.y1, O.y1};
    const Rect c = {O.x0, I.x0, I.y0, I.y1}, e = {I.x1, O.x1, I.y0, I.y1};
    auto pairs = [&](const Rect &R) {
        return vec && !R.empty() && ((R.x0 - par) & 1) == 0 && (R.w() & 1) == 0;
    };
    const bool ta = pairs(a), tb = pairs(b), tc = pairs(c), te = pairs(e);
    const int wa = ta ? a.w() >> 1 : a.w(), wb = tb ? b.w() >> 1 : b.w();
    const int wc = tc ? c.w() >> 1 : c.w(), we = te ? e.w() >> 1 : e.w();
    const int s1 = wa * a.h(), s2 = s1 + wb * b.h(), s3 = s2 + wc * c.h();
    const int total = s3 + we * e.h();
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        // the branches pick coordinates only: f has one call site
        int x, y;
        bool two;
        if (q < s1) {
            x = a.x0 + (q % wa) * (ta ? 2 : 1);
            y = a.y0 + q / wa;
            two = ta;
        } else if (q < s2) {
            const int r = q - s1;
            x = b.x0 + (r % wb) * (tb ? 2 : 1);
            y = b.y0 + r / wb;
            two = tb;
        } else if (q < s3) {
            const int r = q - s2;
            x = c.x0 + (r % wc) * (tc ? 2 : 1);
            y = c.y0 + r / wc;
            two = tc;
        } else {
            const int r = q - s3;
            x = e.x0 + (r % we) * (te ? 2 : 1);
            y = e.y0 + r / we;
            two = te;
        }
        f(x, y, two);
    }
}

// Visit R with the CTA's threads two horizontally adjacent cells (x, x+1)
// per thread (f gets two = true) when R is an even number of cells wide,
// else one cell per thread.
template <class F>
__device__ __forceinline__ void for_pairs(Rect R, F &&f)
{
    const int w = R.w(), h = R.h();
    const bool two = (w & 1) == 0;
    const int wu = two ? w >> 1 : w;
    const int total = wu * h;
    for (int q = threadIdx.x; q < total; q += blockDim.x)
        f(R.x0 + (q % wu) * (two ? 2 : 1), R.y0 + q / wu, two);
}

template <class F>
__device__ __forceinline__ void for_rect(Rect R, F &&f)
{
    const int w = R.w(), total = R.area();
    for (int q = threadIdx.x; q < total; q += blockDim.x)
        f(R.x0 + q % w, R.y0 + q / w);
}


// Index of the window cell (x, y) of the window at (ox, oy) inside one
// component plane of a level-store slot.  The store keeps each 2 x 2 block
// of cells together (32 bytes: one DRAM sector), blocks row-major, so that
// the thin column pieces of the frames and rings that shapes hand over fill
// whole sectors; a row-major store would fetch and write a sector for every
// 8 or 16 bytes of such a column.  nx and ny are even.
// The pieces are 2n cells thick.  For n = 2 they start on even coordinates
// at every level; for n = 1 a piece of level l starts on coordinates of l's
// parity (d and b/2 even), so odd levels of a one-cell-radius equation shift
// the block grid by one cell (shift = 1) to keep the pieces block-aligned.
__device__ __forceinline__ int64_t sidx(const Params &p, int64_t ox, int64_t oy, int x, int y,
                                        int shift)
{
    if (p.narrow) {  // the same arithmetic in 32 bits
        const int nx = (int)p.nx, ny = (int)p.ny;
        int gx = (int)ox + x + shift, gy = (int)oy + y + shift;
        if (gx < 0) gx += nx;
        if (gx >= nx) gx -= nx;
        if (gy < 0) gy += ny;
        if (gy >= ny) gy -= ny;
        return (int64_t)((((gy >> 1) * (nx >> 1) + (gx >> 1)) << 2) + ((gy & 1) << 1) + (gx & 1));
    }
    int64_t gx = ox + x + shift, gy = oy + y + shift;
    if (gx < 0) gx += p.nx;
    if (gx >= p.nx) gx -= p.nx;
    if (gy < 0) gy += p.ny;
    if (gy >= p.ny) gy -= p.ny;
    return (((gy >> 1) * (p.nx >> 1) + (gx >> 1)) << 2) + ((gy & 1) << 1) + (gx & 1);
}

// Asynchronous global -> shared copies (cp.async): 16 bytes cached in L2
// only (.cg), or 8 bytes; and the wait for all of this thread's copies.
// Both addresses of a 16-byte copy are 16-byte aligned.
__device__ __forceinline__ void cp_async16(double *smem_dst, const double *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(double *smem_dst, const double *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// copy one unit of for_units (two cells when `two`, both addresses 16-byte
// aligned; else one) between two places with plain loads and stores
__device__ __forceinline__ void copy_unit(double *dst, const double *src, bool two)
{
    if (two)
        *reinterpret_cast<double2 *>(dst) = *reinterpret_cast<const double2 *>(src);
    else
        *dst = *src;
}

// Whether a window's shared-memory pairs can be 16-byte aligned: an even
// origin ox (always, for a block edge that is a multiple of 4) and an even
// pitch wp (always for the swept windows; a Standard block edge could be
// odd).  Otherwise every copy takes the one-cell path.
template <class EQ, int C>
__device__ __forceinline__ bool pairs_ok(const Block<EQ, C> &B)
{
    return ((B.ox | B.wp) & 1) == 0;
}

// Level-store traffic of one CTA (loads go to this CTA's copy only).  A
// piece's pairs start on the global column parity of the store's blocks,
// i.e. window column (ox + shift) mod 2.
template <class EQ, int C>
__device__ __forceinline__ void load_level_async(const Params &p, Block<EQ, C> &B, int64_t level,
                                                 Rect O, Rect I)
{
    const double *src = B.slot(p, level);
    double *dst = B.lev(level);
    const int64_t gplane = p.nx * p.ny;
    const int shift = EQ::N == 1 ? (int)(level & 1) : 0;
    const int par = (int)((B.ox + shift) & 1);
    for_units(O, I, par, pairs_ok(B), [&](int x, int y, bool two) {
        const int64_t g = sidx(p, B.ox, B.oy, x, y, shift);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c) {
            double *d = dst + c * B.plane + y * B.wp + x;
            if (two)
                cp_async16(d, src + c * gplane + g);
            else
                cp_async8(d, src + c * gplane + g);
        }
    });
}

template <class EQ, int C>
__device__ __forceinline__ void store_level(const Params &p, Block<EQ, C> &B, int64_t level, Rect O,
                                            Rect I)
{
    double *dst = B.slot(p, level);
    const double *src = B.lev(level);
    const int64_t gplane = p.nx * p.ny;
    const int shift = EQ::N == 1 ? (int)(level & 1) : 0;
    const int par = (int)((B.ox + shift) & 1);
    for_units(O, I, par, pairs_ok(B), [&](int x, int y, bool two) {
        const int64_t g = sidx(p, B.ox, B.oy, x, y, shift);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            copy_unit(dst + c * gplane + g, src + c * B.plane + y * B.wp + x, two);
    });
}

// A whole rectangle R of the window between the row-major state (global,
// periodic) and buffer `buf` of shared memory, in 16-byte pairs of cells
// (x, x+1), x even, where pairs_ok holds and the buffer has no one-double
// offset (a pair never straddles the periodic seam: nx is even); one cell at
// a time otherwise.  to_smem: state -> shared memory, else shared memory ->
// state, where `check` (set for the launch that writes a run's final state:
// an infinity or a NaN anywhere in a run reaches it) reports non-finite
// values in the device error word.
template <class EQ, int C>
__device__ __forceinline__ void state_rect(const Params &p, Block<EQ, C> &B, double *state, int buf,
                                           Rect R, bool to_smem, bool check = false)
{
    const int64_t gplane = p.nx * p.ny;
    double *sm = buf ? B.buf[1] : B.buf[0];
    const bool vec = pairs_ok(B) && (buf == 0 || Block<EQ, C>::kHoff == 0);
    bool bad = false;
    for_units(R, Rect{0, 0, 0, 0}, 0, vec, [&](int x, int y, bool two) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c) {
            double *s = sm + c * B.plane + y * B.wp + x;
            double *d = state + c * gplane + g;
            if (to_smem) {
                copy_unit(s, d, two);
            } else {
                copy_unit(d, s, two);
                if (check)
                    bad = bad || nonfinite(s[0]) || (two && nonfinite(s[1]));
            }
        }
    });
    if (bad)
        report(p, kErrNonFinite);
}

// -------------------------------------------------------------- stage kernels

// Advance this CTA's band of region R to `level` (RK2: odd levels are first
// stages, even levels second stages).  Reads buf[(level-1)&1] on the band
// grown by n, and for a second stage the cell's own value two levels back,
// which sits in buf[level&1].  Results go to every CTA of the cluster; the
// caller ends the level with level_barrier<C>().
template <class EQ, int C>
struct Stage;

template <int C>
struct Stage<Heat, C> {
    __device__ __forceinline__ static void run(const Params &p, Block<Heat, C> &B, int64_t level,
                                               Rect R)
    {
        const bool second = (level & 1) == 0;
        const double *src = B.lev(level - 1);
        const double *own = second ? B.lev(level) : src;
        const double c = second ? p.c2 : p.c1;
        const int wp = B.wp;
        for_rect(band(R, B.rank, C), [&](int x, int y) {
            const int i = y * wp + x;
            B.put(level, 0, i,
                  heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp], own[i], c,
                              p.ek.f));
        });
    }
    // Two neighbouring cells per thread (two independent FP64 chains that
    // hide each other's latency, half the index arithmetic per cell) wherever
    // the region is an even number of cells wide, else one.
    __device__ __forceinline__ static void run_pairs(const Params &p, Block<Heat, C> &B,
                                                     int64_t level, Rect R)
    {
        const bool second = (level & 1) == 0;
        const double *src = B.lev(level - 1);
        const double *own = second ? B.lev(level) : src;
        const double c = second ? p.c2 : p.c1;
        const int wp = B.wp;
        for_pairs(band(R, B.rank, C), [&](int x, int y, bool two) {
            const int i = y * wp + x;
            const double a = heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp],
                                         own[i], c, p.ek.f);
            if (two) {
                const double e = heat_update(src[i + 1], src[i], src[i + 2], src[i + 1 - wp],
                                             src[i + 1 + wp], own[i + 1], c, p.ek.f);
                B.put(level, 0, i + 1, e);
            }
            B.put(level, 0, i, a);
        });
    }
    // The swept kernels' form on large grids: one cell per thread, and two
    // neighbouring cells per thread only on levels of at least 16 cells per
    // thread (the full-window levels of b = 64).  Measured at heat 16384^2,
    // Swept Gcell-steps/s against that threshold: 2: 47.7, 4: 50.2, 8: 50.8,
    // 12: 51.3, 16: 51.9, never taken: 51.9; and 49.2 for the same one-cell
    // loop with no pair branch at all.  The branch's presence changes how
    // the compiler lays out the one-cell loop, which carries nearly every
    // level; the arithmetic and its order are the same in all of them.
    __device__ __forceinline__ static void run_wide(const Params &p, Block<Heat, C> &B,
                                                    int64_t level, Rect R)
    {
        const bool second = (level & 1) == 0;
        const double *src = B.lev(level - 1);
        const double *own = second ? B.lev(level) : src;
        const double c = second ? p.c2 : p.c1;
        const int wp = B.wp;
        const Rect S = band(R, B.rank, C);
        if (S.area() >= 16 * (int)blockDim.x && (S.w() & 1) == 0) {
            pairs(p, B, level, S, src, own, c);
            return;
        }
        for_rect(S, [&](int x, int y) {
            const int i = y * wp + x;
            B.put(level, 0, i,
                  heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp], own[i], c,
                              p.ek.f));
        });
    }
    // cells (x, x+1) of an even-width region S, one pair per thread
    __device__ __forceinline__ static void pairs(const Params &p, Block<Heat, C> &B, int64_t level,
                                                 Rect S, const double *src, const double *own,
                                                 double c)
    {
        const int wp = B.wp;
        const int wu = S.w() >> 1, total = wu * S.h();
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            const int i = (S.y0 + q / wu) * wp + S.x0 + 2 * (q % wu);
            const double a = heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp],
                                         own[i], c, p.ek.f);
            const double e = heat_update(src[i + 1], src[i], src[i + 2], src[i + 1 - wp],
                                         src[i + 1 + wp], own[i + 1], c, p.ek.f);
            B.put(level, 0, i, a);
            B.put(level, 0, i + 1, e);
        }
    }
};

template <int C>
struct Stage<HeatFE, C> {
    __device__ __forceinline__ static void run(const Params &p, Block<HeatFE, C> &B, int64_t level,
                                               Rect R)
    {
        const double *src = B.lev(level - 1);
        const int wp = B.wp;
        for_rect(band(R, B.rank, C), [&](int x, int y) {
            const int i = y * wp + x;
            B.put(level, 0, i,
                  heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp], src[i], p.c2,
                              p.ek.f));
        });
    }
};

// One Euler stage (App. B) over this CTA's band of a region: cell
// pressures, half limiter factors, face fluxes, conservative update.  EQ is
// Euler or EulerHist; HIST (EulerHist) also writes every computed level to
// the level history of Params.
template <class EQ, int C, bool HIST>
struct EulerStage {
    __device__ __forceinline__ static void run(const Params &p, Block<EQ, C> &B, int64_t level,
                                               Rect R)
    {
        const int np = B.bands / C;
        for (int k = 0; k < np; ++k) {
            if (k) __syncthreads();  // the scratch of the previous sub-band is free
            run_band(p, B, level, band(R, B.rank * np + k, B.bands));
        }
    }
    __device__ __forceinline__ static void run_band(const Params &p, Block<EQ, C> &B, int64_t level,
                                                    Rect S)
    {
        const bool second = (level & 1) == 0;
        const double *src = B.lev(level - 1);
        const double *own = second ? B.lev(level) : src;
        const double lam = second ? p.c2 : p.c1;
        const int wp = B.wp, pl = B.plane;
        const EulerConst k = p.ek;
        const bool idle = S.empty();
        const int ya = S.y0;
        // scratch row origins
        const int py0 = ya - 2;  // P rows [ya-2, yb+2)
        const int hy0 = ya - 1;  // HY rows [ya-1, yb+1)

        // Each phase below walks one index space over all its items, and the
        // branches on the index pick addresses only: the FP64 body has a
        // single call site, so a warp that straddles two parts of the space
        // does not run it once per part (every FP64 warp instruction costs
        // the same issue time however few of its lanes are active).
        //
        // (a) cell pressures: 2 rows below S and 2 above (S's columns), then
        //     S's rows widened by 2 on each side
        if (!idle) {
            const int W = S.w(), band2 = 2 * W, wide = W + 4;
            const int total = 2 * band2 + wide * S.h();
            for (int q = threadIdx.x; q < total; q += blockDim.x) {
                int x, y;
                if (q < band2) {
                    x = S.x0 + q % W;
                    y = S.y0 - 2 + q / W;
                } else if (q < 2 * band2) {
                    const int r = q - band2;
                    x = S.x0 + r % W;
                    y = S.y1 + r / W;
                } else {
                    const int r = q - 2 * band2;
                    x = S.x0 - 2 + r % wide;
                    y = S.y0 + r / wide;
                }
                const int i = y * wp + x;
                B.P[(y - py0) * wp + x] =
                    cell_pressure(src[i], src[pl + i], src[2 * pl + i], src[3 * pl + i], k);
            }
        }
        __syncthreads();
        // (b) half limiter factors: x on [x0-1, x1+1) x S.rows, y on S.cols x [ya-1, yb+1)
        if (!idle) {
            const Rect lx = {S.x0 - 1, S.x1 + 1, S.y0, S.y1};
            const Rect ly = {S.x0, S.x1, S.y0 - 1, S.y1 + 1};
            const int nlx = lx.area(), total = nlx + ly.area();
            for (int q = threadIdx.x; q < total; q += blockDim.x) {
                int j, st;
                double *hp, *hm;
                if (q < nlx) {
                    const int x = lx.x0 + q % lx.w(), y = lx.y0 + q / lx.w();
                    j = (y - py0) * wp + x;
                    st = 1;
                    const int o = (y - ya) * wp + x;
                    hp = B.hxp + o;
                    hm = B.hxm + o;
                } else {
                    const int r = q - nlx;
                    const int x = ly.x0 + r % ly.w(), y = ly.y0 + r / ly.w();
                    j = (y - py0) * wp + x;
                    st = wp;
                    const int o = (y - hy0) * wp + x;
                    hp = B.hyp + o;
                    hm = B.hym + o;
                }
                const double pc = B.P[j];
                limiter_halves(fadd(pc, -B.P[j - st], k.f), fadd(B.P[j + st], -pc, k.f), p.literal,
                               k.f, *hp, *hm);
            }
        }
        __syncthreads();
        // (c) face fluxes: x faces f = x0..x1 on S's rows (between f-1 and f),
        //     y faces g = ya..yb on S's columns (between g-1 and g); a y face
        //     takes its states in the y-normal frame (rho, m_y, m_x, E), that
        //     is components 2 and 1 swapped on the way in and on the way out
        const int W = S.w(), Hh = S.h();
        const int fxw = W + 1;
        const int nfx = fxw * Hh;
        const int nfy = W * (Hh + 1);
        const int rows = band_rows(wp, Euler::N, B.bands);
        const int fxpl = rows * (wp - 3);        // x-flux component plane
        const int fypl = (rows + 1) * (wp - 4);  // y-flux component plane
        if (!idle) {
            // face q: its left cell's index, the stride to the right cell,
            // the frame's component order, the limiter halves and the output
            auto face = [&](int q, int &i0, int &st, int &ca, int &cb, int &opl, const double *&hl,
                            const double *&hr, double *&out) {
                if (q < nfx) {
                    const int fo = q % fxw, yo = q / fxw;
                    const int x = S.x0 + fo, y = S.y0 + yo;
                    i0 = y * wp + x - 1;
                    st = 1;
                    ca = 1;
                    cb = 2;
                    const int h0 = yo * wp + x - 1;
                    hl = B.hxp + h0;
                    hr = B.hxm + h0 + 1;
                    out = B.fx + yo * fxw + fo;
                    opl = fxpl;
                } else {
                    const int r = q - nfx;
                    const int xo = r % W, go = r / W;
                    const int x = S.x0 + xo, y = S.y0 + go;
                    i0 = (y - 1) * wp + x;
                    st = wp;
                    ca = 2;
                    cb = 1;
                    const int h0 = (y - 1 - hy0) * wp + x;
                    hl = B.hyp + h0;
                    hr = B.hym + h0 + wp;
                    out = B.fy + go * W + xo;
                    opl = fypl;
                }
            };
            // Faces past the last whole group of 128 (one warp per SM
            // sub-partition) cost a whole face's FP64 issue time however few
            // they are.  When at most 64 are left they go two lanes per face
            // (face_flux_half), onto the warps after the last full pass.
            const int total = nfx + nfy;
            const int rem = total & 127;
            const int nsplit = (rem != 0 && rem <= 64) ? rem : 0;
            const int nnorm = total - nsplit;
            for (int q = threadIdx.x; q < nnorm; q += blockDim.x) {
                int i0, st, ca, cb, opl;
                const double *hl, *hr;
                double *out;
                face(q, i0, st, ca, cb, opl, hl, hr, out);
                const int i1 = i0 + st;
                const double q0[4] = {src[i0], src[ca * pl + i0], src[cb * pl + i0], src[3 * pl + i0]};
                const double q1[4] = {src[i1], src[ca * pl + i1], src[cb * pl + i1], src[3 * pl + i1]};
                double fh[4];
                face_flux(q0, q1, *hl, *hr, k, fh);
                out[0] = fh[0];
                out[ca * opl] = fh[1];
                out[cb * opl] = fh[2];
                out[3 * opl] = fh[3];
            }
            if (nsplit) {
                // nnorm is a multiple of 128: the lanes start at a warp
                // boundary, after the threads of the last normal pass
                const int l = (int)threadIdx.x - (int)(nnorm % blockDim.x);
                const bool part = l >= 0 && l < 2 * nsplit;
                const unsigned mask = __ballot_sync(0xffffffffu, part);
                if (part) {
                    int i0, st, ca, cb, opl;
                    const double *hl, *hr;
                    double *out;
                    face(nnorm + (l >> 1), i0, st, ca, cb, opl, hl, hr, out);
                    const int i1 = i0 + st;
                    const double q0[4] = {src[i0], src[ca * pl + i0], src[cb * pl + i0],
                                          src[3 * pl + i0]};
                    const double q1[4] = {src[i1], src[ca * pl + i1], src[cb * pl + i1],
                                          src[3 * pl + i1]};
                    const int side = l & 1;
                    double fa, fb;
                    face_flux_half(q0, q1, *hl, *hr, side, mask, k, fa, fb);
                    out[(side ? cb : 0) * opl] = fa;
                    out[(side ? 3 : ca) * opl] = fb;
                }
            }
        }
        __syncthreads();
        // (d) conservative update of S, written to every CTA of the cluster
        //     (and to the level history, where one is recorded)
        if (!idle) {
            double *hist = nullptr;
            if constexpr (HIST) {
                if (level < p.hist_levels)
                    hist = (level & 1) ? p.hist_qs + ((level - 1) >> 1) * p.hist_stride
                                       : p.hist_q + (level >> 1) * p.hist_stride;
            }
            const int64_t gplane = p.nx * p.ny;
            for_rect(S, [&](int x, int y) {
                const int i = y * wp + x;
                const int xo = x - S.x0, yo = y - S.y0;
                const int ofx = yo * fxw + xo;  // face at x - 1/2
                const int ofy = yo * W + xo;    // face at y - 1/2
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double v =
                        euler_combine(B.fx[c * fxpl + ofx], B.fx[c * fxpl + ofx + 1],
                                      B.fy[c * fypl + ofy], B.fy[c * fypl + ofy + W],
                                      own[c * pl + i], lam, k.f);
                    B.put(level, c, i, v);
                    if constexpr (HIST) {
                        if (hist) hist[c * gplane + gidx(p, B.ox, B.oy, x, y)] = v;
                    }
                }
            });
            (void)hist;
            (void)gplane;
        }
    }
};

template <int C>
struct Stage<Euler, C> : EulerStage<Euler, C, false> {};

template <int C>
struct Stage<EulerHist, C> : EulerStage<EulerHist, C, true> {};

// -------------------------------------------------------------- shape engines

enum ShapeKind { kUp = 0, kXBridge = 1, kYBridge = 2, kLower = 3 };

__device__ __forceinline__ Rect shape_rect(int kind, int b, int n, int s)
{
    const int h = b / 2;
    switch (kind) {
    case kUp: return {s * n, b - s * n, s * n, b - s * n};
    case kXBridge: return {h - s * n, h + s * n, s * n, b - s * n};
    case kYBridge: return {s * n, b - s * n, h - s * n, h + s * n};
    default: return {h - s * n, h + s * n, h - s * n, h + s * n};
    }
}

// The part of level base+s of a shape that other shapes read: the 2n-wide
// frame of an Up-Pyramid level, the two 2n-wide bands of a Bridge level that
// face the neighbouring corners, the whole top level of either.  Returned as
// O \ I.
__device__ __forceinline__ void export_part(int kind, int n, int s, int d, Rect R, Rect &O, Rect &I)
{
    O = R;
    I = {0, 0, 0, 0};
    if (s == d || kind == kLower)
        return;
    const int w = 2 * n;
    if (kind == kUp)
        I = {R.x0 + w, R.x1 - w, R.y0 + w, R.y1 - w};
    else if (kind == kXBridge)
        I = {R.x0, R.x1, R.y0 + w, R.y1 - w};
    else
        I = {R.x0 + w, R.x1 - w, R.y0, R.y1};
    if (I.empty())
        I = {0, 0, 0, 0};
}

// export the part of the level computed by this CTA (its band of R)
template <class EQ, int C>
__device__ __forceinline__ void export_band(const Params &p, Block<EQ, C> &B, int kind, int s,
                                            int64_t level, Rect R)
{
    Rect O, I;
    export_part(kind, EQ::N, s, p.d, R, O, I);
    const Rect S = band(R, B.rank, C);
    const Rect Oc = clip_rows(O, S.y0, S.y1);
    Rect Ic = I.empty() ? I : clip_rows(I, S.y0, S.y1);
    if (Ic.empty())
        Ic = {0, 0, 0, 0};
    store_level(p, B, level, Oc, Ic);
}

// One level of a swept shape.  WIDE (heat on large grids, the host's
// choice): Stage::run_wide, whose levels of at least 16 cells per thread
// take two cells per thread.
template <class EQ, int C, bool WIDE>
__device__ __forceinline__ void stage(const Params &p, Block<EQ, C> &B, int64_t level, Rect R)
{
    if constexpr (WIDE)
        Stage<EQ, C>::run_wide(p, B, level, R);
    else
        Stage<EQ, C>::run(p, B, level, R);
}

// Everything a growing shape (Bridges, the lower half of an Octahedron)
// needs from other shapes was written by earlier launches, so it is fetched
// at once when the kernel starts: the ring of level base+s-1 around the shape
// at level s, for every s, and for an Octahedron also level base+d outside its
// lower half (the base of its upper half).  Each value goes to the buffer of
// its level's parity at its own cell; no two of them share a cell, and none
// sits where a level computed before its use is written (the rings of one
// parity grow outwards, the computed regions stay inside them).
template <class EQ, int C>
__device__ __forceinline__ void preload_growing(const Params &p, Block<EQ, C> &B, int kind,
                                                int64_t base, bool top)
{
    const int n = EQ::N, b = p.b, d = p.d;
    Rect prev = {0, 0, 0, 0};
    for (int s = 1; s <= d; ++s) {
        const Rect R = shape_rect(kind, b, n, s);
        load_level_async(p, B, base + s - 1, grow(R, n), prev);
        prev = R;
    }
    if (top)
        load_level_async(p, B, base + d, Rect{0, b, 0, b}, shape_rect(kLower, b, n, d));
    cp_async_wait_all();
    __syncthreads();
}

// A shape that grows from nothing, its inputs already preloaded.
template <class EQ, int C, bool WIDE>
__device__ __forceinline__ void run_growing(const Params &p, Block<EQ, C> &B, int kind, int64_t base)
{
    const int n = EQ::N, b = p.b, d = p.d;
    for (int s = 1; s <= d; ++s) {
        const int64_t level = base + s;
        const Rect R = shape_rect(kind, b, n, s);
        stage<EQ, C, WIDE>(p, B, level, R);
        level_barrier<C>();
        if (kind != kLower)
            export_band(p, B, kind, s, level, R);
    }
}

// An Up-Pyramid on the window whose level `base` is already in buffer F of
// every CTA of the cluster.
template <class EQ, int C, bool WIDE>
__device__ __forceinline__ void run_pyramid(const Params &p, Block<EQ, C> &B, int64_t base)
{
    const int n = EQ::N, b = p.b, d = p.d;
    export_band(p, B, kUp, 0, base, shape_rect(kUp, b, n, 0));
    for (int s = 1; s <= d; ++s) {
        const int64_t level = base + s;
        const Rect R = shape_rect(kUp, b, n, s);
        stage<EQ, C, WIDE>(p, B, level, R);
        level_barrier<C>();
        export_band(p, B, kUp, s, level, R);
    }
}

// ------------------------------------------------------------------- kernels
// Grids: one cluster of C consecutive CTAs per shape.

// Up-Pyramid on block (I, J) of the unshifted grid; level 0 is the state.
template <class EQ, int C, bool WIDE = false>
__global__ void __launch_bounds__(EQ::SWEPT_THREADS, 1) k_up(const __grid_constant__ Params p)
{
    extern __shared__ __align__(16) double smem[];
    const unsigned tiles = (unsigned)(p.tiles_x * p.tiles_y);
    if (!launch_ok(p, tiles * C, EQ::SWEPT_THREADS, smem_bytes<EQ>(p.b, C * p.passes)))
        return;
    Block<EQ, C> B;
    B.carve(smem, p.b, p.passes);
    const int t = blockIdx.x / C;
    const int I = t % p.tiles_x, J = t / p.tiles_x;
    B.ox = (int64_t)I * p.b;
    B.oy = (int64_t)J * p.b;
    B.set_levels(p, 0);
    state_rect(p, B, p.state, 0, Rect{0, p.b, 0, p.b}, true);
    level_barrier<C>();  // also: every CTA of the cluster has started
    run_pyramid<EQ, C, WIDE>(p, B, 0);
    level_barrier<C>();  // no CTA leaves while a peer may still write to it
}

// X- and Y-Bridges on the seams of the grid with offset o; shape 2t is the
// X-Bridge right of block t, shape 2t+1 the Y-Bridge above it.
template <class EQ, int C, bool WIDE = false>
__global__ void __launch_bounds__(EQ::SWEPT_THREADS, 1) k_bridges(const __grid_constant__ Params p, int64_t base, int o)
{
    extern __shared__ __align__(16) double smem[];
    const unsigned tiles = (unsigned)(p.tiles_x * p.tiles_y);
    if (!launch_ok(p, 2 * tiles * C, EQ::SWEPT_THREADS, smem_bytes<EQ>(p.b, C * p.passes)))
        return;
    Block<EQ, C> B;
    B.carve(smem, p.b, p.passes);
    const int sh = blockIdx.x / C;
    const int t = sh >> 1, kind = (sh & 1) ? kYBridge : kXBridge;
    const int I = t % p.tiles_x, J = t / p.tiles_x;
    const int h = p.b / 2;
    B.ox = (int64_t)I * p.b + o + (kind == kXBridge ? h : 0);
    B.oy = (int64_t)J * p.b + o + (kind == kYBridge ? h : 0);
    if (B.ox >= p.nx) B.ox -= p.nx;
    if (B.oy >= p.ny) B.oy -= p.ny;
    B.set_levels(p, base);
    preload_growing<EQ, C>(p, B, kind, base, false);
    if constexpr (C > 1) cg::this_cluster().sync();
    run_growing<EQ, C, WIDE>(p, B, kind, base);
    if constexpr (C > 1) cg::this_cluster().sync();
}

// Octahedron at the upper-right corner of block (I, J) of the grid with
// offset o (window = the block of the shifted grid centred on that corner).
// last != 0 makes it the Down-Pyramid: the lower half only, after which the
// window, now complete at level base+d, is written to the state.
template <class EQ, int C, bool WIDE = false>
__global__ void __launch_bounds__(EQ::SWEPT_THREADS, 1) k_octahedron(const __grid_constant__ Params p, int64_t base, int o, int last)
{
    extern __shared__ __align__(16) double smem[];
    const unsigned tiles = (unsigned)(p.tiles_x * p.tiles_y);
    if (!launch_ok(p, tiles * C, EQ::SWEPT_THREADS, smem_bytes<EQ>(p.b, C * p.passes)))
        return;
    Block<EQ, C> B;
    B.carve(smem, p.b, p.passes);
    const int t = blockIdx.x / C;
    const int I = t % p.tiles_x, J = t / p.tiles_x;
    const int h = p.b / 2;
    B.ox = (int64_t)I * p.b + o + h;
    B.oy = (int64_t)J * p.b + o + h;
    if (B.ox >= p.nx) B.ox -= p.nx;
    if (B.oy >= p.ny) B.oy -= p.ny;
    B.set_levels(p, base);
    preload_growing<EQ, C>(p, B, kLower, base, true);
    if constexpr (C > 1) cg::this_cluster().sync();
    run_growing<EQ, C, WIDE>(p, B, kLower, base);
    const int64_t top = base + p.d;
    const Rect whole = {0, p.b, 0, p.b};
    if (!last) {
        run_pyramid<EQ, C, WIDE>(p, B, top);
    } else {
        state_rect(p, B, p.state, (int)(top & 1), band(whole, B.rank, C), false, true);
    }
    if constexpr (C > 1) cg::this_cluster().sync();
}

// One RK2 step of the Standard solver: block (I, J) of edge T = std_tile
// loads its tile plus a 2n halo, takes stage 1 on the tile plus an n halo
// and stage 2 on the tile, and writes the tile to dst (and, if qstar is
// not null, the tile's first-stage values to qstar).  PAIRS (heat only):
// each thread takes two neighbouring cells of a stage (Stage::run_pairs),
// the host's choice for large grids.  THREADS: threads per CTA (the host
// gives 64-wide heat blocks twice the default).
template <class EQ, bool PAIRS = false, int THREADS = EQ::STD_THREADS>
__global__ void __launch_bounds__(THREADS) k_standard(const __grid_constant__ Params p, const double *src, double *dst,
                                                       double *qstar)
{
    extern __shared__ __align__(16) double smem[];
    const int T = p.std_tile, n = EQ::N, wp = T + 4 * n;
    if (!launch_ok(p, (unsigned)p.std_blocks, THREADS, smem_bytes<EQ>(wp, 1)))
        return;
    Block<EQ, 1> B;
    B.carve(smem, wp);
    const int I = blockIdx.x % p.std_tx, J = blockIdx.x / p.std_tx;
    B.ox = (int64_t)I * T - 2 * n;
    B.oy = (int64_t)J * T - 2 * n;
    state_rect(p, B, const_cast<double *>(src), 0, Rect{0, wp, 0, wp}, true);
    __syncthreads();
    if constexpr (PAIRS)
        Stage<EQ, 1>::run_pairs(p, B, 1, {n, wp - n, n, wp - n});
    else
        Stage<EQ, 1>::run(p, B, 1, {n, wp - n, n, wp - n});
    __syncthreads();
    const Rect tile = {2 * n, wp - 2 * n, 2 * n, wp - 2 * n};
    if (qstar)
        state_rect(p, B, qstar, 1, tile, false);
    if constexpr (PAIRS)
        Stage<EQ, 1>::run_pairs(p, B, 2, tile);
    else
        Stage<EQ, 1>::run(p, B, 2, tile);
    __syncthreads();
    state_rect(p, B, dst, 0, tile, false, p.check_out != 0);
}

// One level on every cell (tiles of std_tile with a halo of n): the first
// RK2 stage (rebuilt for the adjoint), or one forward-Euler step.
template <class EQ>
__global__ void __launch_bounds__(EQ::STD_THREADS) k_level1(const __grid_constant__ Params p, const double *src, double *dst)
{
    extern __shared__ __align__(16) double smem[];
    const int T = p.std_tile, n = EQ::N, wp = T + 2 * n;
    if (!launch_ok(p, (unsigned)p.std_blocks, EQ::STD_THREADS, smem_bytes<EQ>(wp, 1)))
        return;
    Block<EQ, 1> B;
    B.carve(smem, wp);
    const int I = blockIdx.x % p.std_tx, J = blockIdx.x / p.std_tx;
    B.ox = (int64_t)I * T - n;
    B.oy = (int64_t)J * T - n;
    state_rect(p, B, const_cast<double *>(src), 0, Rect{0, wp, 0, wp}, true);
    __syncthreads();
    Stage<EQ, 1>::run(p, B, 1, {n, wp - n, n, wp - n});
    __syncthreads();
    state_rect(p, B, dst, 1, Rect{n, wp - n, n, wp - n}, false, p.check_out != 0);
}

}  // namespace sweep
