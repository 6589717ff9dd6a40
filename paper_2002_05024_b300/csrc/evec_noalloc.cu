// evec_noalloc.cu -- evec_standard_noalloc: the robust eigenvector solve
// (no back-transformation) for small matrices, with every byte of scratch
// taken from one fixed array that lives in the library's device image.
//
// Who needs it: callers that must not allocate GPU memory while they run --
// a serving process whose memory pool owns the whole device, code inside a
// region where a cudaMalloc would synchronise the device or fail, or a host
// program with a fixed, pre-reserved memory budget.  The regular entry
// points keep their workspace in a handle that grows with cudaMalloc; this
// one allocates nothing: no cudaMalloc / cudaFree, no pinned host buffers,
// no handle, and its host-side plan lives on the stack.
//
// The scratch array is a file-scope static __device__ array: every GPU that
// loads the library holds it (kScratchBytes) until the process exits.  Host
// code cannot use the array's name as a device address (on the host it is a
// stand-in symbol), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device.  Every call shares the array and leaves its contents behind;
// the status word is cleared at the start of each call and everything else
// is written before it is read.  Calls are serialised on the host and each
// call synchronises its stream before returning (also when it fails after
// queuing work), so calls made through this entry point do not overlap; work on the same device that is launched by
// other means while such a call runs must not touch the array (only this
// file can name it).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/evec.h"
#include "evec_internal.cuh"

namespace evec {

void launch_gather_diagonals(const double *T, int64_t ldt, int64_t n, double *out,
                             cudaStream_t st);
void launch_tile_norms(const double *T, int64_t ldt, const Plan &p, double *tau,
                       double *blk_tau, DevStatus *status, cudaStream_t st, int lower = 1);
int launch_diag_solve(int s, const double *T, int64_t ldt, const Plan &p,
                       const int32_t *tile_start_h, const int32_t *tile_real_h,
                       const int32_t *tile_cplx_h,
                       const double *tau, const double *blk_tau, double *Y, int64_t ldy,
                       int32_t *seg_e, double *seg_nu, int32_t *seg_dx, int32_t *seg_dy,
                       cudaStream_t st, const Pencil *pen = nullptr, bool rhs = false,
                       bool decide = true, int *sms = nullptr);
void launch_tile_update(int s, const double *T, int64_t ldt, const Plan &p, int max_tile,
                        const int32_t *tile_col_h, double *Y, int64_t ldy,
                        const int32_t *seg_dx, const int32_t *seg_dy, double *seg_nu,
                        cudaStream_t st);
void launch_finalize(const Plan &p, double *Y, int64_t ldy, const int32_t *seg_e,
                     int32_t *scale_exp, cudaStream_t st);

namespace {

constexpr int kMaxN = EVEC_NOALLOC_MAX_N;
constexpr int kMaxTiles = kMaxN / 15 + 2;          // tiles of >= 15 rows (tile >= 16)
constexpr size_t kScratchBytes = EVEC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Fixed-capacity host plan (the same layout rules as the regular planner:
// blocks from the subdiagonal, greedy tiles never splitting a 2x2 block,
// units in block order).
struct SmallPlan {
    int n, m, ntiles, nblk, nunits, max_tile;
    int32_t tile_start[kMaxTiles + 1], tile_blk[kMaxTiles + 1];
    int32_t tile_unit[kMaxTiles + 1], tile_col[kMaxTiles + 1];
    int32_t blk_start[kMaxN], unit_col[kMaxN], unit_blk[kMaxN], unit_tile[kMaxN];
    int32_t col_unit[kMaxN];
    int32_t ord_real[kMaxN], ord_cplx[kMaxN], tile_real[kMaxTiles + 1], tile_cplx[kMaxTiles + 1];
    int nreal, ncplx;
    int8_t blk_size[kMaxN], second[kMaxN];
    double unit_lam[2 * kMaxN], unit_own[4 * kMaxN];
    double diag[3 * kMaxN];
};

evec_status plan_small(SmallPlan &P, int n, const uint8_t *sel, int nb, int64_t ldt,
                       int64_t *bad) {
    const double *d = P.diag, *sub = P.diag + n, *sup = P.diag + 2 * n - 1;
    for (int i = 0; i < n; i++) {
        const double v[3] = {d[i], i + 1 < n ? sub[i] : 0.0, i + 1 < n ? sup[i] : 0.0};
        const int64_t idx[3] = {i + i * ldt, (i + 1) + i * ldt, i + (i + 1) * ldt};
        for (int k = 0; k < 3; k++) {
            if (!isfinite(v[k])) { if (bad) *bad = idx[k]; return EVEC_ENONFINITE; }
            if (fabs(v[k]) > kInputMax) { if (bad) *bad = idx[k]; return EVEC_EINVAL; }
        }
    }
    P.nblk = 0;
    for (int i = 0; i < n; i++) P.second[i] = 0;
    for (int i = 0; i < n;) {
        int bs = 1;
        if (i + 1 < n && sub[i] != 0.0) {
            if (i + 2 < n && sub[i + 1] != 0.0) { if (bad) *bad = i + 1; return EVEC_ENOTSCHUR; }
            const double b = sup[i], c = sub[i];
            if (d[i] != d[i + 1] || !((b > 0.0 && c < 0.0) || (b < 0.0 && c > 0.0))) {
                if (bad) *bad = i;
                return EVEC_ENOTSCHUR;
            }
            bs = 2;
            P.second[i + 1] = 1;
        }
        P.blk_start[P.nblk] = i;
        P.blk_size[P.nblk] = (int8_t)bs;
        P.nblk++;
        i += bs;
    }
    P.ntiles = 0;
    P.tile_start[0] = 0;
    P.max_tile = 0;
    while (P.tile_start[P.ntiles] < n) {
        int b = P.tile_start[P.ntiles] + nb;
        if (b >= n) b = n;
        else if (P.second[b]) b -= 1;
        P.max_tile = b - P.tile_start[P.ntiles] > P.max_tile ? b - P.tile_start[P.ntiles] : P.max_tile;
        P.tile_start[++P.ntiles] = b;
    }
    P.nunits = 0;
    P.m = 0;
    int t = 0;
    P.tile_blk[0] = P.tile_unit[0] = P.tile_col[0] = 0;
    for (int k = 0; k < P.nblk; k++) {
        while (P.blk_start[k] >= P.tile_start[t + 1]) {
            t++;
            P.tile_blk[t] = k;
            P.tile_unit[t] = P.nunits;
            P.tile_col[t] = P.m;
        }
        const int p = P.blk_start[k], bs = P.blk_size[k];
        if (!(sel == nullptr || sel[p] || (bs == 2 && sel[p + 1]))) continue;
        const int u = P.nunits++;
        P.unit_col[u] = P.m;
        P.unit_blk[u] = k;
        P.unit_tile[u] = t;
        double *own = &P.unit_own[4 * u];
        if (bs == 1) {
            P.unit_lam[2 * u] = d[p];
            P.unit_lam[2 * u + 1] = 0.0;
            own[0] = 1.0; own[1] = 0.0; own[2] = 0.0; own[3] = 0.0;
        } else {
            const double b = sup[p], c = sub[p];
            const double w = sqrt(fabs(b)) * sqrt(fabs(c));
            P.unit_lam[2 * u] = d[p];
            P.unit_lam[2 * u + 1] = w;
            if (fabs(b) >= fabs(c)) { own[0] = 1.0; own[1] = 0.0; own[2] = 0.0; own[3] = w / b; }
            else { own[0] = -w / c; own[1] = 0.0; own[2] = 0.0; own[3] = 1.0; }
        }
        for (int j = 0; j < bs; j++) P.col_unit[P.m + j] = u;
        P.m += bs;
    }
    for (int tt = t + 1; tt <= P.ntiles; tt++) {
        P.tile_blk[tt] = P.nblk;
        P.tile_unit[tt] = P.nunits;
        P.tile_col[tt] = P.m;
    }
    P.nreal = P.ncplx = 0;
    for (int u = 0; u < P.nunits; u++) {
        if (P.unit_lam[2 * u + 1] == 0.0) P.ord_real[P.nreal++] = u;
        else P.ord_cplx[P.ncplx++] = u;
    }
    int ir = 0, ic = 0;
    for (int tt = 0; tt <= P.ntiles; tt++) {
        while (ir < P.nreal && P.unit_tile[P.ord_real[ir]] < tt) ir++;
        while (ic < P.ncplx && P.unit_tile[P.ord_cplx[ic]] < tt) ic++;
        P.tile_real[tt] = ir;
        P.tile_cplx[tt] = ic;
    }
    return EVEC_OK;
}

// Carve the scratch array; returns the bytes needed (0 offsets when base is
// null: a dry run that only sizes the layout).
struct Layout {
    size_t status, diag, plan, tau, blk_tau, seg_e, seg_dx, seg_dy, seg_nu, end;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// An error after work was queued on st: wait for that work (it may still
// write the shared array) and clear the error, so the lock is released only
// once nothing of this call runs any more.
evec_status drain_and_fail(cudaStream_t st) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return EVEC_ECUDA;
}

Layout layout(int n, int ntiles, int nblk, int nunits, int m) {
    Layout L;
    size_t o = 0;
    L.status = o; o = align_up(o + sizeof(DevStatus), 256);
    L.diag = o; o = align_up(o + sizeof(double) * (3 * (size_t)n), 256);
    L.plan = o;
    const size_t plan_bytes = sizeof(double) * (6 * (size_t)nunits) +
                              sizeof(int32_t) * (6 * (size_t)(ntiles + 1) + nblk + 4 * (size_t)nunits + m) +
                              (size_t)nblk + 64;
    o = align_up(o + plan_bytes, 256);
    L.tau = o; o = align_up(o + sizeof(double) * (size_t)ntiles * ntiles, 256);
    L.blk_tau = o; o = align_up(o + sizeof(double) * (size_t)nblk, 256);
    const size_t segs = (size_t)ntiles * (size_t)m;
    L.seg_e = o; o = align_up(o + 4 * segs, 256);
    L.seg_dx = o; o = align_up(o + 4 * segs, 256);
    L.seg_dy = o; o = align_up(o + 4 * segs, 256);
    L.seg_nu = o; o = align_up(o + 8 * segs, 256);
    L.end = o;
    return L;
}

}  // namespace
}  // namespace evec

using namespace evec;

extern "C" evec_status evec_standard_noalloc(int64_t n, const double *T, int64_t ldt,
                                             const uint8_t *select_host, double *X, int64_t ldx,
                                             int32_t *scale_exp, int tile, void *cuda_stream,
                                             int64_t *bad_index) {
    if (bad_index) *bad_index = -1;
    if (n < 0 || ldt < (n > 0 ? n : 1) || ldx < (n > 0 ? n : 1)) return EVEC_EINVAL;
    const int nb = tile ? tile : 64;
    if (nb < 16 || nb > kMaxTile) return EVEC_EINVAL;
    if (n > kMaxN) return EVEC_ECAPACITY;
    if (n == 0) return EVEC_OK;
    if (!T || !X || !scale_exp) return EVEC_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> guard(g_lock);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return EVEC_ECUDA;
    }
    // once per device, with that device current: the array's device address
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return EVEC_ECUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[dev];

    SmallPlan P;   // host plan on the stack (about 60 KB at n = 512)
    // the diagonals: gathered into the scratch array, read back to the stack
    const size_t diag_off = layout((int)n, 1, 1, 1, 1).diag;
    launch_gather_diagonals(T, ldt, n, (double *)(base + diag_off), st);
    if (cudaGetLastError() != cudaSuccess) return drain_and_fail(st);
    if (cudaMemcpyAsync(P.diag, base + diag_off, sizeof(double) * (3 * (size_t)n - 2),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return drain_and_fail(st);
    evec_status ps = plan_small(P, (int)n, select_host, nb, ldt, bad_index);
    if (ps != EVEC_OK) return ps;
    if (P.m == 0) return EVEC_OK;
    const Layout L = layout((int)n, P.ntiles, P.nblk, P.nunits, P.m);
    if (L.end > kScratchBytes) return EVEC_ECAPACITY;
    if (L.diag != diag_off) return EVEC_ECUDA;   // layout invariant

    // pack the plan on the stack, copy it into the scratch array
    alignas(8) unsigned char packed[sizeof(double) * 6 * kMaxN +
                                    sizeof(int32_t) * (6 * (kMaxTiles + 1) + 6 * kMaxN) +
                                    kMaxN + 64];
    size_t off = 0;
    Plan dp{};
    auto put = [&](const void *src, size_t bytes, size_t align) -> const void * {
        off = align_up(off, align);
        memcpy(packed + off, src, bytes);
        const void *dst = base + L.plan + off;
        off += bytes;
        return dst;
    };
    dp.n = n;
    dp.m = P.m;
    dp.ntiles = P.ntiles;
    dp.nblk = P.nblk;
    dp.nunits = P.nunits;
    dp.nb = nb;
    dp.unit_lam = (const double *)put(P.unit_lam, 16 * (size_t)P.nunits, 8);
    dp.unit_own = (const double *)put(P.unit_own, 32 * (size_t)P.nunits, 8);
    dp.tile_start = (const int32_t *)put(P.tile_start, 4 * (size_t)(P.ntiles + 1), 4);
    dp.tile_blk = (const int32_t *)put(P.tile_blk, 4 * (size_t)(P.ntiles + 1), 4);
    dp.tile_unit = (const int32_t *)put(P.tile_unit, 4 * (size_t)(P.ntiles + 1), 4);
    dp.tile_col = (const int32_t *)put(P.tile_col, 4 * (size_t)(P.ntiles + 1), 4);
    dp.blk_start = (const int32_t *)put(P.blk_start, 4 * (size_t)P.nblk, 4);
    dp.unit_col = (const int32_t *)put(P.unit_col, 4 * (size_t)P.nunits, 4);
    dp.unit_blk = (const int32_t *)put(P.unit_blk, 4 * (size_t)P.nunits, 4);
    dp.unit_tile = (const int32_t *)put(P.unit_tile, 4 * (size_t)P.nunits, 4);
    dp.col_unit = (const int32_t *)put(P.col_unit, 4 * (size_t)P.m, 4);
    dp.nreal = P.nreal;
    dp.ncplx = P.ncplx;
    dp.ord_real = (const int32_t *)put(P.ord_real, 4 * (size_t)P.nreal, 4);
    dp.ord_cplx = (const int32_t *)put(P.ord_cplx, 4 * (size_t)P.ncplx, 4);
    dp.tile_real = (const int32_t *)put(P.tile_real, 4 * (size_t)(P.ntiles + 1), 4);
    dp.tile_cplx = (const int32_t *)put(P.tile_cplx, 4 * (size_t)(P.ntiles + 1), 4);
    dp.blk_size = (const int8_t *)put(P.blk_size, (size_t)P.nblk, 1);

    DevStatus *status = (DevStatus *)(base + L.status);
    dp.status = status;
    double *tau = (double *)(base + L.tau);
    double *blk_tau = (double *)(base + L.blk_tau);
    int32_t *seg_e = (int32_t *)(base + L.seg_e);
    int32_t *seg_dx = (int32_t *)(base + L.seg_dx);
    int32_t *seg_dy = (int32_t *)(base + L.seg_dy);
    double *seg_nu = (double *)(base + L.seg_nu);

    // the status word is the only scratch that must start at zero
    if (cudaMemsetAsync(status, 0, sizeof(DevStatus), st) != cudaSuccess ||
        cudaMemcpyAsync(base + L.plan, packed, off, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return drain_and_fail(st);
    launch_tile_norms(T, ldt, dp, tau, blk_tau, status, st);
    for (int s = P.ntiles - 1; s >= 0; s--) {
        launch_diag_solve(s, T, ldt, dp, P.tile_start, P.tile_real, P.tile_cplx, tau, blk_tau, X,
                          ldx, seg_e,
                          seg_nu, seg_dx, seg_dy, st);
        if (s > 0 && P.tile_col[s] < P.m)
            launch_tile_update(s, T, ldt, dp, P.max_tile, P.tile_col, X, ldx, seg_dx, seg_dy,
                               seg_nu, st);
    }
    launch_finalize(dp, X, ldx, seg_e, scale_exp, st);
    if (cudaGetLastError() != cudaSuccess) return drain_and_fail(st);
    DevStatus hs;
    if (cudaMemcpyAsync(&hs, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return drain_and_fail(st);
    if (hs.code != 0 && bad_index) *bad_index = hs.index;
    return (evec_status)hs.code;
}
