// kernels.cuh -- swept-rule phase kernels and the Standard step kernel.
//
// Geometry (Sec. 3.3; levels are RK stages, n the radius of one stage, b the
// block edge, d the levels one phase advances, 2 <= d <= b/(2n) - 1 (Eq. 1),
// d even).  Every kernel below gives one CTA a b x b window of the periodic
// grid and takes one shape through its levels inside shared memory:
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
// reads and writes only cells of its own window, and the windows of one
// launch partition the plane, so no two CTAs of a launch touch the same word
// of a slot.  Within the CTA the full-step levels live in buffer F and the
// stage levels in buffer H; a second stage updates F in place.
#pragma once

#include <cstdint>

#include "numerics.cuh"

namespace sweep {

constexpr int kThreads = 256;

struct Rect {
    int x0, x1, y0, y1;
    __device__ __forceinline__ int w() const { return x1 > x0 ? x1 - x0 : 0; }
    __device__ __forceinline__ int h() const { return y1 > y0 ? y1 - y0 : 0; }
    __device__ __forceinline__ int area() const { return w() * h(); }
    __device__ __forceinline__ bool empty() const { return x1 <= x0 || y1 <= y0; }
};

__device__ __forceinline__ Rect grow(Rect r, int g) { return {r.x0 - g, r.x1 + g, r.y0 - g, r.y1 + g}; }

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
};

// ------------------------------------------------------------------ equations

struct Heat {
    static constexpr int NC = 1;
    static constexpr int N = 1;
};
struct Euler {
    static constexpr int NC = 4;
    static constexpr int N = 2;
};

// shared-memory bytes of one CTA with window edge wp
template <class EQ>
__host__ __device__ constexpr size_t smem_bytes(int wp)
{
    if (EQ::NC == 1)
        return sizeof(double) * 2 * (size_t)wp * wp;
    // F, H (4 comps each), P, four limiter halves, x and y face fluxes
    return sizeof(double) * ((size_t)8 * wp * wp + (size_t)wp * wp + (size_t)4 * wp * wp +
                             (size_t)8 * wp * (wp + 1));
}

// Per-CTA view of shared memory.
template <class EQ>
struct Block {
    double *buf[2];  // F (even levels), H (odd levels): [NC][wp*wp]
    double *P;       // Euler: cell pressure [wp*wp]
    double *hxp, *hxm, *hyp, *hym;  // Euler: half limiter factors [wp*wp]
    double *fx, *fy;                // Euler: face fluxes [4][wp*(wp+1)]
    int wp;          // window pitch (edge)
    int64_t ox, oy;  // global origin of the window
    int plane;       // wp*wp

    __device__ void carve(double *smem, int wp_)
    {
        wp = wp_;
        plane = wp * wp;
        buf[0] = smem;
        buf[1] = smem + EQ::NC * plane;
        double *p = smem + 2 * EQ::NC * plane;
        if (EQ::NC == 4) {
            P = p;
            p += plane;
            hxp = p;
            p += plane;
            hxm = p;
            p += plane;
            hyp = p;
            p += plane;
            hym = p;
            p += plane;
            fx = p;
            p += 4 * wp * (wp + 1);
            fy = p;
        }
    }
};

__device__ __forceinline__ int64_t gidx(const Params &p, int64_t ox, int64_t oy, int x, int y)
{
    int64_t gx = ox + x, gy = oy + y;
    // windows start inside [0, n) and extend at most one grid period
    if (gx < 0) gx += p.nx;
    if (gx >= p.nx) gx -= p.nx;
    if (gy < 0) gy += p.ny;
    if (gy >= p.ny) gy -= p.ny;
    return gy * p.nx + gx;
}

// Visit every cell of O \ I (I inside O or empty) with the CTA's threads,
// packed linearly so that no lane idles while work is left.
template <class F>
__device__ __forceinline__ void for_diff(Rect O, Rect I, F &&f)
{
    Rect part[4];
    int np = 0;
    if (O.empty())
        return;
    if (I.empty()) {
        part[np++] = O;
    } else {
        part[np++] = {O.x0, O.x1, O.y0, I.y0};  // below I
        part[np++] = {O.x0, O.x1, I.y1, O.y1};  // above I
        part[np++] = {O.x0, I.x0, I.y0, I.y1};  // left of I
        part[np++] = {I.x1, O.x1, I.y0, I.y1};  // right of I
    }
    int total = 0;
    for (int k = 0; k < np; ++k)
        total += part[k].area();
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        int r = q, k = 0;
        while (r >= part[k].area()) {
            r -= part[k].area();
            ++k;
        }
        const int w = part[k].w();
        f(part[k].x0 + r % w, part[k].y0 + r / w);
    }
}

template <class F>
__device__ __forceinline__ void for_rect(Rect R, F &&f)
{
    const int w = R.w(), total = R.area();
    for (int q = threadIdx.x; q < total; q += blockDim.x)
        f(R.x0 + q % w, R.y0 + q / w);
}

__device__ __forceinline__ double *slot_ptr(const Params &p, int64_t level)
{
    return p.ws + (level % (p.d + 1)) * p.slot_elems;
}

// level-store traffic of one CTA
template <class EQ>
__device__ __forceinline__ void load_level(const Params &p, Block<EQ> &B, int64_t level, Rect O,
                                           Rect I)
{
    const double *src = slot_ptr(p, level);
    double *dst = B.buf[level & 1];
    const int64_t gplane = p.nx * p.ny;
    for_diff(O, I, [&](int x, int y) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            dst[c * B.plane + y * B.wp + x] = src[c * gplane + g];
    });
}

template <class EQ>
__device__ __forceinline__ void store_level(const Params &p, Block<EQ> &B, int64_t level, Rect O,
                                            Rect I)
{
    double *dst = slot_ptr(p, level);
    const double *src = B.buf[level & 1];
    const int64_t gplane = p.nx * p.ny;
    for_diff(O, I, [&](int x, int y) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            dst[c * gplane + g] = src[c * B.plane + y * B.wp + x];
    });
}

// -------------------------------------------------------------- stage kernels

// Advance region R to `level` (RK2: odd levels are first stages, even levels
// second stages).  Reads buf[(level-1)&1] on R grown by n, and for a second
// stage the cell's own value two levels back, which sits in buf[level&1].
template <class EQ>
__device__ void stage_region(const Params &p, Block<EQ> &B, int64_t level, Rect R);

template <>
__device__ void stage_region<Heat>(const Params &p, Block<Heat> &B, int64_t level, Rect R)
{
    const bool second = (level & 1) == 0;
    const double *src = B.buf[(level - 1) & 1];
    double *dst = B.buf[level & 1];
    const double *own = second ? dst : src;
    const double c = second ? p.c2 : p.c1;
    const int wp = B.wp;
    for_rect(R, [&](int x, int y) {
        const int i = y * wp + x;
        dst[i] = heat_update(src[i], src[i - 1], src[i + 1], src[i - wp], src[i + wp], own[i], c);
    });
}

template <>
__device__ void stage_region<Euler>(const Params &p, Block<Euler> &B, int64_t level, Rect R)
{
    const bool second = (level & 1) == 0;
    const double *src = B.buf[(level - 1) & 1];
    double *dst = B.buf[level & 1];
    const double *own = second ? dst : src;
    const double lam = second ? p.c2 : p.c1;
    const int wp = B.wp, pl = B.plane;
    const EulerConst k = p.ek;
    if (R.empty())
        return;

    // (a) cell pressures on the cross R (+-2 in x on R's rows, +-2 in y on R's columns)
    {
        const Rect rx = {R.x0 - 2, R.x1 + 2, R.y0, R.y1};
        const Rect ry = {R.x0, R.x1, R.y0 - 2, R.y1 + 2};
        for_diff(ry, R, [&](int x, int y) {
            const int i = y * wp + x;
            B.P[i] = cell_pressure(src[i], src[pl + i], src[2 * pl + i], src[3 * pl + i], k);
        });
        for_rect(rx, [&](int x, int y) {
            const int i = y * wp + x;
            B.P[i] = cell_pressure(src[i], src[pl + i], src[2 * pl + i], src[3 * pl + i], k);
        });
    }
    __syncthreads();
    // (b) half limiter factors: x on [x0-1, x1+1) x R.y, y on R.x x [y0-1, y1+1)
    {
        const Rect lx = {R.x0 - 1, R.x1 + 1, R.y0, R.y1};
        const Rect ly = {R.x0, R.x1, R.y0 - 1, R.y1 + 1};
        const int nlx = lx.area(), total = nlx + ly.area();
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            if (q < nlx) {
                const int x = lx.x0 + q % lx.w(), y = lx.y0 + q / lx.w();
                const int i = y * wp + x;
                const double pc = B.P[i];
                limiter_halves(__dadd_rn(pc, -B.P[i - 1]), __dadd_rn(B.P[i + 1], -pc), p.literal,
                               B.hxp[i], B.hxm[i]);
            } else {
                const int r = q - nlx;
                const int x = ly.x0 + r % ly.w(), y = ly.y0 + r / ly.w();
                const int i = y * wp + x;
                const double pc = B.P[i];
                limiter_halves(__dadd_rn(pc, -B.P[i - wp]), __dadd_rn(B.P[i + wp], -pc),
                               p.literal, B.hyp[i], B.hym[i]);
            }
        }
    }
    __syncthreads();
    // (c) face fluxes: x faces f = x0..x1 on each row (between f-1 and f),
    //     y faces g = y0..y1 on each column (between g-1 and g)
    const int W = R.w(), Hh = R.h();
    const int fxw = W + 1;           // x faces per row
    const int nfx = fxw * Hh;        // x faces
    const int nfy = W * (Hh + 1);    // y faces
    const int fpl = wp * (wp + 1);   // face-array plane
    {
        const int total = nfx + nfy;
        for (int q = threadIdx.x; q < total; q += blockDim.x) {
            double fh[4];
            if (q < nfx) {
                const int fo = q % fxw, yo = q / fxw;
                const int x = R.x0 + fo, y = R.y0 + yo;
                const int i0 = y * wp + x - 1, i1 = i0 + 1;
                const double q0[4] = {src[i0], src[pl + i0], src[2 * pl + i0], src[3 * pl + i0]};
                const double q1[4] = {src[i1], src[pl + i1], src[2 * pl + i1], src[3 * pl + i1]};
                face_flux(q0, q1, B.hxp[i0], B.hxm[i1], k, fh);
                const int o = yo * fxw + fo;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    B.fx[c * fpl + o] = fh[c];
            } else {
                const int r = q - nfx;
                const int xo = r % W, go = r / W;
                const int x = R.x0 + xo, y = R.y0 + go;
                const int i0 = (y - 1) * wp + x, i1 = i0 + wp;
                // y-normal frame: (rho, m_y, m_x, E)
                const double q0[4] = {src[i0], src[2 * pl + i0], src[pl + i0], src[3 * pl + i0]};
                const double q1[4] = {src[i1], src[2 * pl + i1], src[pl + i1], src[3 * pl + i1]};
                face_flux(q0, q1, B.hyp[i0], B.hym[i1], k, fh);
                const int o = go * W + xo;
                B.fy[o] = fh[0];
                B.fy[fpl + o] = fh[2];
                B.fy[2 * fpl + o] = fh[1];
                B.fy[3 * fpl + o] = fh[3];
            }
        }
    }
    __syncthreads();
    // (d) conservative update of R
    for_rect(R, [&](int x, int y) {
        const int i = y * wp + x;
        const int xo = x - R.x0, yo = y - R.y0;
        const int ofx = yo * fxw + xo;  // face at x - 1/2
        const int ofy = yo * W + xo;    // face at y - 1/2
#pragma unroll
        for (int c = 0; c < 4; ++c)
            dst[c * pl + i] = euler_combine(B.fx[c * fpl + ofx], B.fx[c * fpl + ofx + 1],
                                            B.fy[c * fpl + ofy], B.fy[c * fpl + ofy + W],
                                            own[c * pl + i], lam);
    });
}

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

// Shapes that grow from nothing (Bridges, the lower half of an Octahedron):
// before each level, fetch from the level store the part of the previous
// level around the shape that other shapes produced.
template <class EQ>
__device__ void run_growing(const Params &p, Block<EQ> &B, int kind, int64_t base)
{
    const int n = EQ::N, b = p.b, d = p.d;
    Rect prev = {0, 0, 0, 0};
    for (int s = 1; s <= d; ++s) {
        const int64_t level = base + s;
        const Rect R = shape_rect(kind, b, n, s);
        load_level(p, B, level - 1, grow(R, n), prev);
        __syncthreads();
        stage_region<EQ>(p, B, level, R);
        __syncthreads();
        if (kind != kLower) {
            Rect O, I;
            export_part(kind, n, s, d, R, O, I);
            store_level(p, B, level, O, I);
        }
        prev = R;
    }
}

// An Up-Pyramid on the window whose level `base` is already in buffer F.
template <class EQ>
__device__ void run_pyramid(const Params &p, Block<EQ> &B, int64_t base)
{
    const int n = EQ::N, b = p.b, d = p.d;
    {
        Rect O, I;
        export_part(kUp, n, 0, d, shape_rect(kUp, b, n, 0), O, I);
        store_level(p, B, base, O, I);
    }
    for (int s = 1; s <= d; ++s) {
        const int64_t level = base + s;
        const Rect R = shape_rect(kUp, b, n, s);
        stage_region<EQ>(p, B, level, R);
        __syncthreads();
        Rect O, I;
        export_part(kUp, n, s, d, R, O, I);
        store_level(p, B, level, O, I);
    }
}

// ------------------------------------------------------------------- kernels

// Up-Pyramid on block (I, J) of the unshifted grid; level 0 is the state.
template <class EQ>
__global__ void __launch_bounds__(kThreads) k_up(Params p)
{
    extern __shared__ double smem[];
    Block<EQ> B;
    B.carve(smem, p.b);
    const int I = blockIdx.x % p.tiles_x, J = blockIdx.x / p.tiles_x;
    B.ox = (int64_t)I * p.b;
    B.oy = (int64_t)J * p.b;
    const int64_t gplane = p.nx * p.ny;
    for_rect({0, p.b, 0, p.b}, [&](int x, int y) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            B.buf[0][c * B.plane + y * B.wp + x] = p.state[c * gplane + g];
    });
    __syncthreads();
    run_pyramid<EQ>(p, B, 0);
}

// X- and Y-Bridges on the seams of the grid with offset o; CTA 2t is the
// X-Bridge right of block t, CTA 2t+1 the Y-Bridge above it.
template <class EQ>
__global__ void __launch_bounds__(kThreads) k_bridges(Params p, int64_t base, int o)
{
    extern __shared__ double smem[];
    Block<EQ> B;
    B.carve(smem, p.b);
    const int t = blockIdx.x >> 1, kind = (blockIdx.x & 1) ? kYBridge : kXBridge;
    const int I = t % p.tiles_x, J = t / p.tiles_x;
    const int h = p.b / 2;
    B.ox = (int64_t)I * p.b + o + (kind == kXBridge ? h : 0);
    B.oy = (int64_t)J * p.b + o + (kind == kYBridge ? h : 0);
    if (B.ox >= p.nx) B.ox -= p.nx;
    if (B.oy >= p.ny) B.oy -= p.ny;
    run_growing<EQ>(p, B, kind, base);
}

// Octahedron at the upper-right corner of block (I, J) of the grid with
// offset o (window = the block of the shifted grid centred on that corner).
// last != 0 makes it the Down-Pyramid: the lower half only, after which the
// window, now complete at level base+d, is written to the state.
template <class EQ>
__global__ void __launch_bounds__(kThreads) k_octahedron(Params p, int64_t base, int o, int last)
{
    extern __shared__ double smem[];
    Block<EQ> B;
    B.carve(smem, p.b);
    const int I = blockIdx.x % p.tiles_x, J = blockIdx.x / p.tiles_x;
    const int h = p.b / 2;
    B.ox = (int64_t)I * p.b + o + h;
    B.oy = (int64_t)J * p.b + o + h;
    if (B.ox >= p.nx) B.ox -= p.nx;
    if (B.oy >= p.ny) B.oy -= p.ny;
    run_growing<EQ>(p, B, kLower, base);
    const int64_t top = base + p.d;
    const Rect whole = {0, p.b, 0, p.b};
    load_level(p, B, top, whole, shape_rect(kLower, p.b, EQ::N, p.d));
    __syncthreads();
    if (!last) {
        run_pyramid<EQ>(p, B, top);
    } else {
        const int64_t gplane = p.nx * p.ny;
        const double *src = B.buf[top & 1];
        for_rect(whole, [&](int x, int y) {
            const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
            for (int c = 0; c < EQ::NC; ++c)
                p.state[c * gplane + g] = src[c * B.plane + y * B.wp + x];
        });
    }
}

// One RK2 step of the Standard solver: block (I, J) of edge T = std_tile
// loads its tile plus a 2n halo, takes stage 1 on the tile plus an n halo
// and stage 2 on the tile, and writes the tile to dst.
template <class EQ>
__global__ void __launch_bounds__(kThreads) k_standard(Params p, const double *src, double *dst)
{
    extern __shared__ double smem[];
    const int T = p.std_tile, n = EQ::N, wp = T + 4 * n;
    Block<EQ> B;
    B.carve(smem, wp);
    const int tx = (int)(p.nx / T);
    const int I = blockIdx.x % tx, J = blockIdx.x / tx;
    B.ox = (int64_t)I * T - 2 * n;
    B.oy = (int64_t)J * T - 2 * n;
    const int64_t gplane = p.nx * p.ny;
    for_rect({0, wp, 0, wp}, [&](int x, int y) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            B.buf[0][c * B.plane + y * wp + x] = src[c * gplane + g];
    });
    __syncthreads();
    stage_region<EQ>(p, B, 1, {n, wp - n, n, wp - n});
    __syncthreads();
    stage_region<EQ>(p, B, 2, {2 * n, wp - 2 * n, 2 * n, wp - 2 * n});
    __syncthreads();
    for_rect({2 * n, wp - 2 * n, 2 * n, wp - 2 * n}, [&](int x, int y) {
        const int64_t g = gidx(p, B.ox, B.oy, x, y);
#pragma unroll
        for (int c = 0; c < EQ::NC; ++c)
            dst[c * gplane + g] = B.buf[0][c * B.plane + y * wp + x];
    });
}

}  // namespace sweep
