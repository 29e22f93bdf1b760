// sweep_api.cu -- the C ABI of include/sweep.h: handle, argument checks,
// workspace sizing and the launch sequences of the Swept and Standard solvers.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <iterator>
#include <type_traits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "adjoint.cuh"
#include "kernels.cuh"
#include "sweep.h"

using namespace sweep;

struct sweep_s {
    int eqn;
    int64_t nx, ny;
    double dt, dx;
    int tile, depth;
    double alpha, gamma;
    int limiter;   // 0 textbook orientation, 1 as printed
    int scheme;    // heat: 0 RK2 midpoint, 1 forward Euler
    int std_tile;
    int cluster;     // CTAs per Up-Pyramid / Octahedron window (1, 2 or 4)
    int cluster_br;  // CTAs per Bridge window (1, 2 or 4)
    int passes;      // sub-bands per CTA and level (1, 2 or 4)
    int check;       // 1: every run ends by reading the device error word (synchronous)
    int l2_fetch;    // L2 fetch granularity this handle set for the context (0: untouched)
    // optional per-launch event timing ("profile" parameter)
    int profile;
    std::vector<cudaEvent_t> ev;   // start/end pairs, reused across runs
    std::vector<int> ev_kind;      // kernel kind of each recorded pair
    size_t ev_used;                // pairs recorded since the last read
};

namespace {

constexpr size_t kHeader = 256;  // workspace header: the device error word, then padding

// ---- host-side fault injection (test hooks; nothing here touches a GPU)
std::atomic<int> fault_site{0};   // armed site, 0 = none
std::atomic<int> fault_count{0};  // passes through the site left before the failure
std::atomic<int> live_objects{0};  // CUDA streams and events the library holds

// true on the pass through `site` that was armed to fail (then disarms)
bool inject(int site)
{
    if (fault_site.load() != site) return false;
    if (fault_count.fetch_sub(1) != 1) return false;
    fault_site.store(0);
    return true;
}

int radius(int eqn) { return eqn == SWEEP_HEAT ? 1 : 2; }
int ncomp(int eqn) { return eqn == SWEEP_HEAT ? 1 : 4; }

int64_t slot_elems(const sweep_s *h)
{
    const int64_t e = (int64_t)ncomp(h->eqn) * h->nx * h->ny;
    return (e + 31) / 32 * 32;  // 256-byte multiple
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

constexpr size_t kMaxSmem = 227 * 1024;
constexpr int64_t kStdMinBlocks = 148;  // SMs of a B300 (Standard blocks, swept CTAs)

// shared-memory bytes of a swept CTA / a Standard CTA
size_t swept_smem(int eqn, int b, int C)
{
    return eqn == SWEEP_HEAT ? smem_bytes<Heat>(b, C) : smem_bytes<Euler>(b, C);
}

bool valid_std_tile(const sweep_s *h, int t)
{
    const int n = radius(h->eqn);
    if (t < 8 || t > 64 || h->nx % t != 0 || h->ny % t != 0) return false;
    return swept_smem(h->eqn, t + 4 * n, 1) <= kMaxSmem;
}

bool valid_cluster(int eqn, int b, int C)
{
    return (C == 1 || C == 2 || C == 4) && swept_smem(eqn, b, C) <= kMaxSmem;
}

bool valid_passes(int P) { return P == 1 || P == 2 || P == 4; }

Params make_params(const sweep_s *h, double *state, void *ws)
{
    Params p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.b = h->tile;
    p.d = h->depth;
    p.tiles_x = (int)(h->nx / h->tile);
    p.tiles_y = (int)(h->ny / h->tile);
    p.std_tile = h->std_tile;
    p.std_tx = (int)(h->nx / h->std_tile);
    p.std_blocks = p.std_tx * (int)(h->ny / h->std_tile);
    if (h->eqn == SWEEP_HEAT) {
        const double r = (h->alpha * h->dt) / (h->dx * h->dx);
        p.c1 = 0.5 * r;
        p.c2 = r;
    } else {
        const double lam = h->dt / h->dx;
        p.c1 = 0.5 * lam;
        p.c2 = lam;
    }
    p.ek.gamma = h->gamma;
    p.ek.gm1 = h->gamma - 1.0;
    p.ek.f.one = 1.0;
    p.ek.f.nzero = -0.0;
    p.literal = h->limiter;
    p.state = state;
    p.ws = ws ? (double *)((char *)ws + kHeader) : nullptr;
    p.slot_elems = slot_elems(h);
    p.passes = h->passes;
    p.hist_q = nullptr;
    p.hist_qs = nullptr;
    p.hist_stride = 0;
    p.hist_levels = 0;
    p.err = ws ? (unsigned *)ws : nullptr;
    p.check_out = 0;
    p.narrow = h->nx * h->ny < (int64_t(1) << 31) ? 1 : 0;
    return p;
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Kernel kinds for the profile counters.
enum { kKindUp = 0, kKindBridges = 1, kKindOctahedron = 2, kKindDown = 3, kKindStandard = 4,
       kKinds = 5 };

// Event bracket around one launch when profiling is on.
struct Bracket {
    sweep_s *h;
    cudaStream_t st;
    size_t i;
    bool on;
    Bracket(const sweep_s *hc, cudaStream_t s, int kind) : h(const_cast<sweep_s *>(hc)), st(s), i(0), on(false)
    {
        if (!h->profile) return;
        i = h->ev_used;
        if (2 * (i + 1) > h->ev.size()) {
            cudaEvent_t a, b;
            if (inject(SWEEP_SITE_EVENTS) || cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) {
                cudaEventDestroy(a);
                return;
            }
            h->ev.push_back(a);
            h->ev.push_back(b);
            h->ev_kind.push_back(kind);
            live_objects += 2;
        }
        h->ev_kind[i] = kind;
        on = cudaEventRecord(h->ev[2 * i], st) == cudaSuccess;
    }
    ~Bracket()
    {
        if (on && cudaEventRecord(h->ev[2 * i + 1], st) == cudaSuccess) h->ev_used = i + 1;
    }
};

// Standard launches over `nlevels` levels: two levels (one RK2 step, or two
// forward-Euler steps) per launch and, for an odd count, one single-level
// launch; ping-pong between the state and slot 0 of the workspace, ending in
// the state.
// the Standard heat step takes two cells per thread on grids of at least
// 2^20 cells (throughput-bound: heat 16384^2 46.5 -> 48.4 Gcell-steps/s),
// one on smaller ones (latency-bound: heat 64^2 1.57 against 1.36)
constexpr int64_t kStdPairsCells = int64_t(1) << 20;
// threads of a 64-wide heat Standard block, paired: 512 (heat 4096^2 47.8 ->
// 49.0 Gcell-steps/s against 256; 16384^2 51.1 either way; 32-wide and
// smaller blocks are fastest at 256)
constexpr int kStdThreads64 = 512;

template <class EQ>
int standard_levels(const sweep_s *h, Params p, int64_t nlevels, cudaStream_t st)
{
    if (nlevels <= 0) return SWEEP_OK;
    const int T = h->std_tile;
    const size_t smem = smem_bytes<EQ>(T + 4 * EQ::N, 1);
    const size_t smem1 = smem_bytes<EQ>(T + 2 * EQ::N, 1);
    void (*step)(Params, const double *, double *, double *) = k_standard<EQ>;
    int threads = EQ::STD_THREADS;
    if constexpr (std::is_same<EQ, Heat>::value)
        if (h->nx * h->ny >= kStdPairsCells) {
            step = k_standard<Heat, true>;
            if (T == 64) {
                step = k_standard<Heat, true, kStdThreads64>;
                threads = kStdThreads64;
            }
        }
    if (set_smem(step, smem) != cudaSuccess || set_smem(k_level1<EQ>, smem1) != cudaSuccess)
        return SWEEP_ECUDA;
    const unsigned grid = (unsigned)((h->nx / T) * (h->ny / T));
    double *a = p.state, *b = p.ws;
    // the launch that writes the run's final state checks it for infinities
    // and NaNs (device error word)
    Params last = p;
    last.check_out = 1;
    for (int64_t l = 0; l + 1 < nlevels; l += 2) {
        {
            Bracket br(h, st, kKindStandard);
            step<<<grid, threads, smem, st>>>(l + 2 >= nlevels ? last : p, a, b, nullptr);
        }
        double *t = a;
        a = b;
        b = t;
    }
    if (nlevels & 1) {
        {
            Bracket br(h, st, kKindStandard);
            k_level1<EQ><<<grid, EQ::STD_THREADS, smem1, st>>>(last, a, b);
        }
        double *t = a;
        a = b;
        b = t;
    }
    if (cudaGetLastError() != cudaSuccess) return SWEEP_ECUDA;
    if (a != p.state) {
        const size_t bytes = sizeof(double) * (size_t)ncomp(h->eqn) * h->nx * h->ny;
        if (cudaMemcpyAsync(p.state, a, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SWEEP_ECUDA;
    }
    return SWEEP_OK;
}

// launch one swept kernel with C-CTA clusters of `threads` threads each
template <int C, class... KArgs, class... Args>
cudaError_t launch(void (*kernel)(KArgs...), unsigned shapes, int threads, size_t smem,
                   cudaStream_t st, Args... args)
{
    if constexpr (C == 1) {
        kernel<<<shapes, threads, smem, st>>>(args...);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(shapes * C, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, args...);
    }
}

template <class EQ, int C, int CB, bool WIDE>
int swept_c(const sweep_s *h, Params p, int64_t nlevels, cudaStream_t st)
{
    const int64_t L = nlevels;
    const int d = h->depth;
    int64_t done = 0;
    if (L >= d) {
        const size_t smem = smem_bytes<EQ>(h->tile, C * h->passes);
        const size_t smem_b = smem_bytes<EQ>(h->tile, CB * h->passes);
        if (set_smem(k_up<EQ, C, WIDE>, smem) != cudaSuccess ||
            set_smem(k_bridges<EQ, CB, WIDE>, smem_b) != cudaSuccess ||
            set_smem(k_octahedron<EQ, C, WIDE>, smem) != cudaSuccess)
            return SWEEP_ECUDA;
        const unsigned tiles = (unsigned)(p.tiles_x * p.tiles_y);
        const int64_t m = L / d - 1;  // whole [Bridges, Octahedron] cycles
        cudaError_t e;
        {
            Bracket br(h, st, kKindUp);
            e = launch<C>(k_up<EQ, C, WIDE>, tiles, EQ::SWEPT_THREADS, smem, st, p);
        }
        for (int64_t c = 0; c <= m && e == cudaSuccess; ++c) {
            const int o = (c & 1) ? h->tile / 2 : 0;
            const int64_t base = c * d;
            {
                Bracket br(h, st, kKindBridges);
                e = launch<CB>(k_bridges<EQ, CB, WIDE>, 2 * tiles, EQ::SWEPT_THREADS, smem_b, st, p,
                               base, o);
            }
            if (e != cudaSuccess) break;
            {
                Bracket br(h, st, c == m ? kKindDown : kKindOctahedron);
                e = launch<C>(k_octahedron<EQ, C, WIDE>, tiles, EQ::SWEPT_THREADS, smem, st, p, base,
                              o, c == m ? 1 : 0);
            }
        }
        if (e != cudaSuccess) return SWEEP_ECUDA;
        done = (m + 1) * d;
    }
    return standard_levels<EQ>(h, p, L - done, st);
}

// Heat on a grid of at least 2^16 cells runs the WIDE swept kernels
// (Stage<Heat>::run_wide: levels of at least 16 cells per thread in pairs).
// Block 64, Gcell-steps/s against the one-cell kernels: heat 16384^2 49.2
// -> 51.9, 768^2 34.5 -> 35.6, 512^2 17.6 -> 17.9, 256^2 4.42 -> 4.49.
// Smaller grids run the one-cell kernels, which the wide form slows by
// 3.5 % at heat 64^2 (0.597 -> 0.576).
constexpr int64_t kSweptWideCells = int64_t(1) << 16;

template <class EQ, int C, int CB>
int swept_w(const sweep_s *h, Params p, int64_t nlevels, cudaStream_t st)
{
    if constexpr (std::is_same<EQ, Heat>::value)
        if (h->nx * h->ny >= kSweptWideCells) return swept_c<EQ, C, CB, true>(h, p, nlevels, st);
    return swept_c<EQ, C, CB, false>(h, p, nlevels, st);
}

template <class EQ, int C>
int swept_b(const sweep_s *h, Params p, int64_t nlevels, cudaStream_t st)
{
    switch (h->cluster_br) {
    case 2: return swept_w<EQ, C, 2>(h, p, nlevels, st);
    case 4: return swept_w<EQ, C, 4>(h, p, nlevels, st);
    default: return swept_w<EQ, C, 1>(h, p, nlevels, st);
    }
}

// swept run over `nlevels` stage-levels (2 per RK2 step, 1 per forward-Euler step)
template <class EQ>
int swept(const sweep_s *h, Params p, int64_t nlevels, cudaStream_t st)
{
    switch (h->cluster) {
    case 2: return swept_b<EQ, 2>(h, p, nlevels, st);
    case 4: return swept_b<EQ, 4>(h, p, nlevels, st);
    default: return swept_b<EQ, 1>(h, p, nlevels, st);
    }
}

bool heat_fe(const sweep_s *h) { return h->eqn == SWEEP_HEAT && h->scheme == 1; }

int run_swept_any(const sweep_s *h, Params p, int64_t nsteps, cudaStream_t st)
{
    if (heat_fe(h)) return swept<HeatFE>(h, p, nsteps, st);
    if (h->eqn == SWEEP_HEAT) return swept<Heat>(h, p, 2 * nsteps, st);
    return swept<Euler>(h, p, 2 * nsteps, st);
}

int run_standard_any(const sweep_s *h, Params p, int64_t nsteps, cudaStream_t st)
{
    if (heat_fe(h)) return standard_levels<HeatFE>(h, p, nsteps, st);
    if (h->eqn == SWEEP_HEAT) return standard_levels<Heat>(h, p, 2 * nsteps, st);
    return standard_levels<Euler>(h, p, 2 * nsteps, st);
}

// ------------------------------------------------------------ adjoint

struct AdjLayout {
    size_t store, ckpt, seg, qs, mu, cp, lp, faces, total;  // byte offsets (after the header)
    int64_t nseg, ckpt_every;
};

AdjLayout adjoint_layout(const sweep_s *h, int64_t nsteps, int64_t ckpt)
{
    AdjLayout L = {};
    const size_t st = sizeof(double) * (size_t)slot_elems(h);
    L.store = 0;
    size_t off = st * (size_t)(h->depth + 1);  // level store of the swept forward
    if (h->eqn == SWEEP_HEAT) {
        L.total = off;
        return L;
    }
    L.ckpt_every = ckpt;
    L.nseg = nsteps > 0 ? (nsteps + ckpt - 1) / ckpt : 0;
    L.ckpt = off;
    off += st * (size_t)(L.nseg > 0 ? L.nseg : 1);
    L.seg = off;
    off += st * (size_t)ckpt;
    L.qs = off;  // first-stage states of the segment
    off += st * (size_t)ckpt;
    L.mu = off;
    off += st;
    const size_t plane = sizeof(double) * (size_t)h->nx * (size_t)h->ny;
    L.cp = off;
    off += (plane * 4 + 255) / 256 * 256;
    L.lp = off;
    off += (plane * 12 + 255) / 256 * 256;
    L.faces = off;
    off += plane * 2 * kFacePlanes;
    L.total = off;
    return L;
}

int euler_adjoint(sweep_s *h, const double *q0, const double *lamT, double *lam0, int64_t nsteps,
                  int64_t ckpt, void *ws, cudaStream_t st)
{
    const AdjLayout L = adjoint_layout(h, nsteps, ckpt);
    char *base = (char *)ws + kHeader;
    const size_t sbytes = sizeof(double) * 4 * (size_t)h->nx * (size_t)h->ny;
    const size_t sstride = sizeof(double) * (size_t)slot_elems(h);
    auto ckpt_ptr = [&](int64_t s) { return (double *)(base + L.ckpt + sstride * (size_t)s); };
    auto seg_ptr = [&](int64_t t) { return (double *)(base + L.seg + sstride * (size_t)t); };
    auto qs_ptr = [&](int64_t t) { return (double *)(base + L.qs + sstride * (size_t)t); };
    double *mu = (double *)(base + L.mu);
    double *cp = (double *)(base + L.cp), *lp = (double *)(base + L.lp);
    double *faces = (double *)(base + L.faces);
    if (cudaMemcpyAsync(lam0, lamT, sbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SWEEP_ECUDA;
    if (nsteps == 0) return SWEEP_OK;
    // forward pass: checkpoints every `ckpt` steps, advanced with the swept solver
    if (cudaMemcpyAsync(ckpt_ptr(0), q0, sbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SWEEP_ECUDA;
    for (int64_t s = 0; s + 1 < L.nseg; ++s) {
        if (cudaMemcpyAsync(ckpt_ptr(s + 1), ckpt_ptr(s), sbytes, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return SWEEP_ECUDA;
        const int rc = swept<Euler>(h, make_params(h, ckpt_ptr(s + 1), ws), 2 * ckpt, st);
        if (rc != SWEEP_OK) return rc;
    }
    // backward pass, segment by segment
    Params p = make_params(h, nullptr, ws);
    const int T = h->std_tile;
    const size_t smem_std = smem_bytes<Euler>(T + 4 * Euler::N, 1);
    if (set_smem(k_standard<Euler>, smem_std) != cudaSuccess) return SWEEP_ECUDA;
    const unsigned tiles = (unsigned)((h->nx / T) * (h->ny / T));
    const int64_t plane = h->nx * h->ny;
    const unsigned gf = (unsigned)((2 * plane + kVjpThreads - 1) / kVjpThreads);
    const unsigned gc = (unsigned)((plane + kThreads - 1) / kThreads);
    for (int64_t s = L.nseg - 1; s >= 0; --s) {
        const int64_t len = (s + 1) * ckpt <= nsteps ? ckpt : nsteps - s * ckpt;
        if (cudaMemcpyAsync(seg_ptr(0), ckpt_ptr(s), sbytes, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return SWEEP_ECUDA;
        // recompute the segment swept-wise from its checkpoint, recording
        // every level: Q^t in seg_ptr(t), the first stages Q*_t in
        // qs_ptr(t); mu (unused yet) holds the running state.  The steps
        // left after the last whole swept cycle are Standard steps that
        // write Q*_t as well; the last step's end state is not needed and
        // lands in mu.
        const int64_t swept_levels = 2 * len >= h->depth ? (2 * len / h->depth) * h->depth : 0;
        if (swept_levels > 0) {
            if (cudaMemcpyAsync(mu, seg_ptr(0), sbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return SWEEP_ECUDA;
            Params ph = make_params(h, mu, ws);
            ph.hist_q = seg_ptr(0);
            ph.hist_qs = qs_ptr(0);
            ph.hist_stride = (int64_t)(sstride / sizeof(double));
            ph.hist_levels = 2 * len;
            const int rc = swept<EulerHist>(h, ph, swept_levels, st);
            if (rc != SWEEP_OK) return rc;
        }
        for (int64_t t = swept_levels / 2; t < len; ++t)
            k_standard<Euler><<<tiles, Euler::STD_THREADS, smem_std, st>>>(
                p, seg_ptr(t), t + 1 < len ? seg_ptr(t + 1) : mu, qs_ptr(t));
        for (int64_t t = len - 1; t >= 0; --t) {
            k_vjp_cells<<<gc, kThreads, 0, st>>>(p, qs_ptr(t), cp);
            k_vjp_limiters<<<gc, kThreads, 0, st>>>(p, cp, lp);
            k_face_vjp<<<gf, kVjpThreads, 0, st>>>(p, qs_ptr(t), lp, lam0, faces);
            k_gather<<<gc, kThreads, 0, st>>>(p, faces, qs_ptr(t), cp, lam0, mu, 0);
            k_vjp_cells<<<gc, kThreads, 0, st>>>(p, seg_ptr(t), cp);
            k_vjp_limiters<<<gc, kThreads, 0, st>>>(p, cp, lp);
            k_face_vjp<<<gf, kVjpThreads, 0, st>>>(p, seg_ptr(t), lp, mu, faces);
            k_gather<<<gc, kThreads, 0, st>>>(p, faces, seg_ptr(t), cp, lam0, mu, 1);
        }
        if (cudaGetLastError() != cudaSuccess) return SWEEP_ECUDA;
    }
    return SWEEP_OK;
}

int check_run(const sweep_t *h, const double *state, int64_t nsteps, const void *ws)
{
    if (!h || !state || !ws || nsteps < 0) return SWEEP_EINVAL;
    if (!aligned(state, 16) || !aligned(ws, 256)) return SWEEP_EINVAL;
    return SWEEP_OK;
}

// clear the device error word before a run's kernels
int clear_error_word(void *ws, cudaStream_t st)
{
    return cudaMemsetAsync(ws, 0, sizeof(unsigned), st) == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

int read_error_word(const void *ws, unsigned *bits, cudaStream_t st)
{
    unsigned w = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(&w, ws, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SWEEP_ECUDA;
    if (bits) *bits = w;
    if (w && cudaMemset(const_cast<void *>(ws), 0, sizeof(unsigned)) != cudaSuccess)
        return SWEEP_ECUDA;
    return w ? SWEEP_EDEVICE : SWEEP_OK;
}

// the end of a run: with "check" on, wait for it and read its error word
int finish_run(const sweep_t *h, int rc, const void *ws, cudaStream_t st)
{
    if (rc != SWEEP_OK || !h->check) return rc;
    return read_error_word(ws, nullptr, st);
}

}  // namespace

extern "C" {
#define SWEEP_API __attribute__((visibility("default")))

SWEEP_API int sweep_create(int eqn, int64_t nx, int64_t ny, double dt, double dx, int tile, int depth,
                 sweep_t **out)
{
    if (!out) return SWEEP_EINVAL;
    *out = nullptr;
    if (eqn != SWEEP_HEAT && eqn != SWEEP_EULER) return SWEEP_EINVAL;
    if (!(std::isfinite(dt) && dt > 0.0 && std::isfinite(dx) && dx > 0.0)) return SWEEP_EINVAL;
    const int n = radius(eqn);
    const int cluster = eqn == SWEEP_HEAT ? 1 : 2;
    if (tile <= 2 * n || (tile % 2) != 0 || !valid_cluster(eqn, tile, cluster)) return SWEEP_EINVAL;
    if (nx <= 0 || ny <= 0 || nx % tile != 0 || ny % tile != 0) return SWEEP_EINVAL;
    if (nx / tile < 2 || ny / tile < 2) return SWEEP_EINVAL;
    if (nx > (int64_t(1) << 31) || ny > (int64_t(1) << 31)) return SWEEP_EINVAL;
    const int k = tile / (2 * n) - 1;  // Eq. 1
    if (depth == 0) depth = k - (k % 2);
    if (depth < 2 || depth > k || (depth % 2) != 0) return SWEEP_EINVAL;
    sweep_s *h = inject(SWEEP_SITE_HOST_ALLOC) ? nullptr : new (std::nothrow) sweep_s;
    if (!h) return SWEEP_ENOMEM;
    h->eqn = eqn;
    h->nx = nx;
    h->ny = ny;
    h->dt = dt;
    h->dx = dx;
    h->tile = tile;
    h->depth = depth;
    h->alpha = 1.0;
    h->gamma = 1.4;
    h->limiter = 0;
    h->scheme = 0;
    h->std_tile = 0;
    // Octahedra of Euler on 2-CTA clusters while the windows' CTAs fit one
    // per SM (at most 74 windows), else on single CTAs; Bridges on single
    // CTAs.  Measured on B300 with 512-thread swept CTAs: vortex 256^2
    // (64 windows) 0.747 Gcell-steps/s with 2-CTA Octahedra; 1024^2 (1024
    // windows) 0.955 with single CTAs against 0.858 with 2-CTA clusters (a
    // 512-thread CTA's registers leave room for one CTA per SM).
    const int64_t windows = (nx / tile) * (ny / tile);
    h->cluster = (cluster == 2 && 2 * windows > kStdMinBlocks && valid_cluster(eqn, tile, 1))
                     ? 1 : cluster;
    h->cluster_br = 1;
    h->passes = 1;
    h->check = 0;
    h->l2_fetch = 0;
    h->profile = 0;
    h->ev_used = 0;
    // Standard block edge: the first preferred edge that cuts the grid into
    // at least its minimum number of blocks, else the allowed edge with the
    // most blocks (a small grid is latency bound: more, smaller blocks finish
    // sooner).  The minimums are measured on B300 (heat, 256^2 to 16384^2):
    // 64- and 32-wide heat blocks pay for their smaller halo share from 1024
    // blocks (64-wide: 2048^2 and up); other edges need one block per SM
    // (148).
    struct Pref {
        int t;
        int64_t min_blocks;
    };
    const Pref heat_prefer[] = {{64, 1024}, {32, 1024}, {16, kStdMinBlocks}, {8, kStdMinBlocks},
                                {24, kStdMinBlocks}, {12, kStdMinBlocks}, {48, kStdMinBlocks},
                                {40, kStdMinBlocks}, {20, kStdMinBlocks}, {10, kStdMinBlocks}};
    const Pref euler_prefer[] = {{16, kStdMinBlocks}, {8, kStdMinBlocks},  {24, kStdMinBlocks},
                                 {12, kStdMinBlocks}, {64, kStdMinBlocks}, {48, kStdMinBlocks},
                                 {40, kStdMinBlocks}, {20, kStdMinBlocks}, {10, kStdMinBlocks}};
    const bool heat = eqn == SWEEP_HEAT;
    const Pref *prefer = heat ? heat_prefer : euler_prefer;
    const int nprefer = heat ? (int)std::size(heat_prefer) : (int)std::size(euler_prefer);
    int64_t most = 0;
    for (int k = 0; k < nprefer; ++k) {
        const Pref &pr = prefer[k];
        const int t = pr.t;
        if (!valid_std_tile(h, t)) continue;
        const int64_t blocks = (nx / t) * (ny / t);
        if (blocks >= pr.min_blocks) {
            h->std_tile = t;
            break;
        }
        if (blocks > most) {
            most = blocks;
            h->std_tile = t;
        }
    }
    // no preferred edge divides the grid (e.g. 56 x 84): the even edge in
    // [8, 64] that gives the most blocks
    for (int t = 8; h->std_tile == 0 && t <= 64; t += 2)
        if (valid_std_tile(h, t)) h->std_tile = t;
    if (h->std_tile == 0) {
        delete h;
        return SWEEP_EINVAL;
    }
    *out = h;
    return SWEEP_OK;
}

SWEEP_API int sweep_set_param(sweep_t *h, const char *key, double v)
{
    if (!h || !key) return SWEEP_EINVAL;
    if (!std::strcmp(key, "alpha")) {
        if (!(std::isfinite(v) && v > 0.0)) return SWEEP_EINVAL;
        h->alpha = v;
    } else if (!std::strcmp(key, "gamma")) {
        if (!(std::isfinite(v) && v > 1.0)) return SWEEP_EINVAL;
        h->gamma = v;
    } else if (!std::strcmp(key, "limiter")) {
        if (v != 0.0 && v != 1.0 && v != 2.0) return SWEEP_EINVAL;
        h->limiter = (int)v;
    } else if (!std::strcmp(key, "scheme")) {
        if (v != 0.0 && v != 1.0) return SWEEP_EINVAL;
        h->scheme = (int)v;
    } else if (!std::strcmp(key, "standard_tile")) {
        if (v != std::floor(v) || !valid_std_tile(h, (int)v)) return SWEEP_EINVAL;
        h->std_tile = (int)v;
    } else if (!std::strcmp(key, "cluster")) {
        if (v != std::floor(v) || !valid_cluster(h->eqn, h->tile, (int)v)) return SWEEP_EINVAL;
        h->cluster = (int)v;
        h->cluster_br = (int)v;
    } else if (!std::strcmp(key, "cluster_oct")) {
        if (v != std::floor(v) || !valid_cluster(h->eqn, h->tile, (int)v)) return SWEEP_EINVAL;
        h->cluster = (int)v;
    } else if (!std::strcmp(key, "cluster_bridges")) {
        if (v != std::floor(v) || !valid_cluster(h->eqn, h->tile, (int)v)) return SWEEP_EINVAL;
        h->cluster_br = (int)v;
    } else if (!std::strcmp(key, "passes")) {
        if (v != std::floor(v) || !valid_passes((int)v)) return SWEEP_EINVAL;
        h->passes = (int)v;
    } else if (!std::strcmp(key, "check")) {
        if (v != 0.0 && v != 1.0) return SWEEP_EINVAL;
        h->check = (int)v;
    } else if (!std::strcmp(key, "l2_fetch_bytes")) {
        if (v != 0.0 && v != 32.0 && v != 64.0 && v != 128.0) return SWEEP_EINVAL;
        if (v != 0.0 &&
            cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)v) != cudaSuccess)
            return SWEEP_ECUDA;
        h->l2_fetch = (int)v;
    } else if (!std::strcmp(key, "profile")) {
        if (v != 0.0 && v != 1.0) return SWEEP_EINVAL;
        h->profile = (int)v;
        h->ev_used = 0;
    } else {
        return SWEEP_EINVAL;
    }
    return SWEEP_OK;
}

SWEEP_API int sweep_get_param(const sweep_t *h, const char *key, double *v)
{
    if (!h || !key || !v) return SWEEP_EINVAL;
    if (!std::strcmp(key, "alpha")) *v = h->alpha;
    else if (!std::strcmp(key, "gamma")) *v = h->gamma;
    else if (!std::strcmp(key, "limiter")) *v = h->limiter;
    else if (!std::strcmp(key, "scheme")) *v = h->scheme;
    else if (!std::strcmp(key, "standard_tile")) *v = h->std_tile;
    else if (!std::strcmp(key, "profile")) *v = h->profile;
    else if (!std::strcmp(key, "check")) *v = h->check;
    else if (!std::strcmp(key, "l2_fetch_bytes")) *v = h->l2_fetch;
    else if (!std::strcmp(key, "cluster") || !std::strcmp(key, "cluster_oct")) *v = h->cluster;
    else if (!std::strcmp(key, "cluster_bridges")) *v = h->cluster_br;
    else if (!std::strcmp(key, "passes")) *v = h->passes;
    else if (!std::strcmp(key, "tile")) *v = h->tile;
    else if (!std::strcmp(key, "depth")) *v = h->depth;
    else if (!std::strcmp(key, "nx")) *v = (double)h->nx;
    else if (!std::strcmp(key, "ny")) *v = (double)h->ny;
    else if (!std::strcmp(key, "ncomp")) *v = ncomp(h->eqn);
    else if (!std::strcmp(key, "radius")) *v = radius(h->eqn);
    else if (!std::strcmp(key, "r")) *v = (h->alpha * h->dt) / (h->dx * h->dx);
    else return SWEEP_EINVAL;
    return SWEEP_OK;
}

SWEEP_API size_t sweep_workspace_bytes(const sweep_t *h)
{
    if (!h) return 0;
    return kHeader + sizeof(double) * (size_t)slot_elems(h) * (size_t)(h->depth + 1);
}

SWEEP_API int sweep_run_swept(sweep_t *h, double *d_state, int64_t nsteps, void *d_ws, CUstream_st *stream)
{
    int rc = check_run(h, d_state, nsteps, d_ws);
    if (rc == SWEEP_OK) rc = clear_error_word(d_ws, stream);
    if (rc != SWEEP_OK) return rc;
    rc = run_swept_any(h, make_params(h, d_state, d_ws), nsteps, stream);
    return finish_run(h, rc, d_ws, stream);
}

SWEEP_API int sweep_run_standard(sweep_t *h, double *d_state, int64_t nsteps, void *d_ws,
                       CUstream_st *stream)
{
    int rc = check_run(h, d_state, nsteps, d_ws);
    if (rc == SWEEP_OK) rc = clear_error_word(d_ws, stream);
    if (rc != SWEEP_OK) return rc;
    rc = run_standard_any(h, make_params(h, d_state, d_ws), nsteps, stream);
    return finish_run(h, rc, d_ws, stream);
}

SWEEP_API size_t sweep_adjoint_workspace_bytes(const sweep_t *h, int64_t nsteps, int ckpt_every)
{
    if (!h || nsteps < 0 || ckpt_every < 1) return 0;
    return kHeader + adjoint_layout(h, nsteps, ckpt_every).total;
}

SWEEP_API int sweep_adjoint(sweep_t *h, const double *d_q0, const double *d_lamT, double *d_lam0,
                            int64_t nsteps, int ckpt_every, void *d_ws, CUstream_st *stream)
{
    if (!h || !d_lamT || !d_lam0 || !d_ws || nsteps < 0 || ckpt_every < 1) return SWEEP_EINVAL;
    if (!aligned(d_lamT, 16) || !aligned(d_lam0, 16) || !aligned(d_ws, 256)) return SWEEP_EINVAL;
    if (h->eqn == SWEEP_EULER && (!d_q0 || !aligned(d_q0, 16) || d_lam0 == d_lamT))
        return SWEEP_EINVAL;
    int rc = clear_error_word(d_ws, stream);
    if (rc != SWEEP_OK) return rc;
    if (h->eqn == SWEEP_HEAT) {
        const size_t bytes = sizeof(double) * (size_t)h->nx * (size_t)h->ny;
        if (d_lam0 != d_lamT &&
            cudaMemcpyAsync(d_lam0, d_lamT, bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
            return SWEEP_ECUDA;
        // the heat step is linear with a symmetric stencil: its adjoint step
        // is a stencil update of the same radius, run swept (the
        // forward-Euler step is its own adjoint)
        if (heat_fe(h))
            rc = swept<HeatFE>(h, make_params(h, d_lam0, d_ws), nsteps, stream);
        else
            rc = swept<HeatAdj>(h, make_params(h, d_lam0, d_ws), 2 * nsteps, stream);
    } else {
        rc = euler_adjoint(h, d_q0, d_lamT, d_lam0, nsteps, ckpt_every, d_ws, stream);
    }
    return finish_run(h, rc, d_ws, stream);
}

SWEEP_API int sweep_check(const void *d_ws, unsigned *bits, CUstream_st *stream)
{
    if (bits) *bits = 0;
    if (!d_ws || !aligned(d_ws, 256)) return SWEEP_EINVAL;
    return read_error_word(d_ws, bits, stream);
}

SWEEP_API int sweep_inject_fault(int site, int nth)
{
    if (nth < 0 || (site != 0 && site != SWEEP_SITE_HOST_ALLOC && site != SWEEP_SITE_STREAM_POOL &&
                    site != SWEEP_SITE_EVENTS))
        return SWEEP_EINVAL;
    fault_site.store(0);
    fault_count.store(nth);
    if (site != 0 && nth > 0) fault_site.store(site);
    return SWEEP_OK;
}

SWEEP_API int sweep_live_cuda_objects(void) { return live_objects.load(); }

// ------------------------------------------------------------------ batch
//
// A batch runs every instance's swept launch sequence on one of a pool of
// internal streams, forked from and joined back into the caller's stream by
// events, so that independent instances overlap on the GPU and the whole
// batch can be captured from the caller's stream into one CUDA graph.

namespace {
constexpr int kBatchStreams = 16;
constexpr int kMaxBatchDevices = 64;
std::mutex batch_mu;
struct BatchPool {
    cudaStream_t s[kBatchStreams];
    cudaEvent_t done[kBatchStreams];
    cudaEvent_t fork;
    bool ready;
};
BatchPool batch_pool[kMaxBatchDevices];

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Create the pool's streams and events.  On a failure everything created so
// far is destroyed again and the pool stays not ready, so a later call
// starts over instead of leaking or reusing half a pool.
int make_batch_pool(BatchPool *bp)
{
    cudaStream_t s[kBatchStreams] = {};
    cudaEvent_t done[kBatchStreams] = {}, fork = nullptr;
    int ns = 0, ne = 0;
    bool ok = true;
    for (int k = 0; k < kBatchStreams && ok; ++k) {
        ok = !inject(SWEEP_SITE_STREAM_POOL) &&
             cudaStreamCreateWithFlags(&s[k], cudaStreamNonBlocking) == cudaSuccess;
        if (ok) ++ns;
        ok = ok && !inject(SWEEP_SITE_STREAM_POOL) &&
             cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming) == cudaSuccess;
        if (ok) ++ne;
    }
    ok = ok && !inject(SWEEP_SITE_STREAM_POOL) &&
         cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (int k = 0; k < ne; ++k) cudaEventDestroy(done[k]);
        for (int k = 0; k < ns; ++k) cudaStreamDestroy(s[k]);
        return SWEEP_ECUDA;
    }
    live_objects += 2 * kBatchStreams + 1;
    for (int k = 0; k < kBatchStreams; ++k) {
        bp->s[k] = s[k];
        bp->done[k] = done[k];
    }
    bp->fork = fork;
    bp->ready = true;
    return SWEEP_OK;
}
}  // namespace

SWEEP_API size_t sweep_batch_workspace_bytes(sweep_t *const *hs, int count)
{
    if (!hs || count < 0) return 0;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return 0;
        total += align256(sweep_workspace_bytes(hs[i]));
    }
    return total;
}

SWEEP_API int sweep_batch_run(sweep_t *const *hs, double *const *d_states, const int64_t *nsteps,
                              int count, void *d_ws, CUstream_st *stream)
{
    if (!hs || !d_states || !nsteps || count < 0 || (count > 0 && !d_ws)) return SWEEP_EINVAL;
    if (!aligned(d_ws, 256)) return SWEEP_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || !d_states[i] || nsteps[i] < 0 || !aligned(d_states[i], 16)) return SWEEP_EINVAL;
    }
    if (count == 0) return SWEEP_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxBatchDevices) return SWEEP_ECUDA;
    BatchPool *bp = &batch_pool[dev];
    {
        std::lock_guard<std::mutex> lock(batch_mu);
        if (!bp->ready) {
            const int rc = make_batch_pool(bp);
            if (rc != SWEEP_OK) return rc;
        }
    }
    // largest work first, dealt round-robin over the streams
    std::vector<int> order(count);
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) {
        order[i] = i;
        cost[i] = (double)hs[i]->nx * (double)hs[i]->ny * (double)nsteps[i] *
                  (hs[i]->eqn == SWEEP_HEAT ? 1.0 : 50.0);
    }
    for (int a = 1; a < count; ++a)
        for (int b = a; b > 0 && cost[order[b - 1]] < cost[order[b]]; --b) {
            const int t = order[b];
            order[b] = order[b - 1];
            order[b - 1] = t;
        }
    std::vector<size_t> off(count);
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        off[i] = o;
        o += align256(sweep_workspace_bytes(hs[i]));
    }
    const int ns = count < kBatchStreams ? count : kBatchStreams;
    if (cudaEventRecord(bp->fork, stream) != cudaSuccess) return SWEEP_ECUDA;
    for (int k = 0; k < ns; ++k)
        if (cudaStreamWaitEvent(bp->s[k], bp->fork, 0) != cudaSuccess) return SWEEP_ECUDA;
    int rc = SWEEP_OK;
    for (int r = 0; r < count && rc == SWEEP_OK; ++r) {
        const int i = order[r];
        rc = sweep_run_swept(hs[i], d_states[i], nsteps[i], (char *)d_ws + off[i], bp->s[r % ns]);
    }
    // join every stream back, even after an error, so no stream is left forked
    for (int k = 0; k < ns; ++k) {
        if (cudaEventRecord(bp->done[k], bp->s[k]) != cudaSuccess ||
            cudaStreamWaitEvent(stream, bp->done[k], 0) != cudaSuccess)
            rc = rc == SWEEP_OK ? SWEEP_ECUDA : rc;
    }
    return rc;
}

SWEEP_API int sweep_profile_read(sweep_t *h, double *ms, int64_t *launches, int nkinds)
{
    if (!h || !ms || !launches || nkinds <= 0) return SWEEP_EINVAL;
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (size_t i = 0; i < h->ev_used; ++i) {
        float t = 0.f;
        if (cudaEventSynchronize(h->ev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess)
            return SWEEP_ECUDA;
        const int k = h->ev_kind[i];
        if (k < nkinds) {
            ms[k] += t;
            launches[k] += 1;
        }
    }
    h->ev_used = 0;
    return SWEEP_OK;
}

SWEEP_API void sweep_destroy(sweep_t *h)
{
    if (!h) return;
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    live_objects -= (int)h->ev.size();
    delete h;
}

SWEEP_API const char *sweep_error_string(int status)
{
    switch (status) {
    case SWEEP_OK: return "ok";
    case SWEEP_EINVAL: return "invalid argument";
    case SWEEP_ENOMEM: return "out of host memory";
    case SWEEP_ECUDA: return "CUDA error";
    case SWEEP_ETIMEOUT: return "device wait timed out";
    case SWEEP_EUNSUPPORTED: return "unsupported";
    case SWEEP_EDEVICE: return "a kernel reported an error (device error word)";
    default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// Allocation-free swept run.
//
// Some callers cannot allocate device memory at the point where they want to
// advance a state: a host application that owns every byte of the GPU through
// its own pool and lets plug-ins allocate nothing, or a timing-critical loop
// in which an allocation (its latency, or its failing halfway through a run)
// is not acceptable.  For them the level store lives in this fixed array
// instead of a caller-provided workspace.  The array exists on every GPU that
// loads this library, for the life of the process.
//
// In host code `sweep_static_scratch` only names a host-side stand-in; its
// device address comes from cudaGetSymbolAddress, taken once per device (with
// that device current) and cached in static_scratch_ptr.
static __device__ __align__(256) unsigned char sweep_static_scratch[SWEEP_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex static_scratch_mu;
void *static_scratch_ptr[kMaxDevices];
}  // namespace

SWEEP_API int sweep_run_swept_static(sweep_t *h, double *d_state, int64_t nsteps,
                                     CUstream_st *stream)
{
    if (!h || !d_state || nsteps < 0 || !aligned(d_state, 16)) return SWEEP_EINVAL;
    if (h->profile) return SWEEP_EUNSUPPORTED;  // profiling creates CUDA events
    if (sweep_workspace_bytes(h) > SWEEP_STATIC_SCRATCH_BYTES) return SWEEP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SWEEP_ECUDA;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(static_scratch_mu);
        if (!static_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, sweep_static_scratch) != cudaSuccess || !p)
                return SWEEP_ECUDA;
            static_scratch_ptr[dev] = p;
        }
        ws = static_scratch_ptr[dev];
    }
    return sweep_run_swept(h, d_state, nsteps, ws, stream);  // clears and, with "check", reads the word
}

}  // extern "C"
