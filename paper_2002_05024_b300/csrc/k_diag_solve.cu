// k_diag_solve.cu -- robust shifted solves on one diagonal tile (Eq. evec_solve
// restricted to the rows of tile s), then the consolidation/protection
// decisions for every tile above it (Sec. 3.3, the preprocessing step of the
// update Z <- Y - T X).
//
// Work split: G lanes per unit -- G = 8 for a real eigenvalue, G = 16 for a
// complex pair solved as one complex column -- and CTAs of W = 4 warps
// (W = 2 for tiles above 64 rows); real and complex units in separate CTAs
// of one launch.  On B300 one SM sub-partition issues at most one FP64
// warp-instruction per 64 cycles, and an FP64 instruction costs that slot
// whether its lanes are active, masked or predicated off, so the FP64
// instructions of a unit's chain are spread thin (a few update rows per
// lane per block step, loop trip counts uniform across the warp) and the W
// warps of a CTA land on different sub-partitions.  Row i of a unit's segment
// belongs to lane i mod G.  The block solves form a sequential chain per
// unit, and a warp issues in order, so the chain is kept short: the
// factors of every shifted 1x1/2x2 block system of the tile are computed
// first (independent of the data, spread over the unit's lanes; pivot
// reciprocals by rcp.approx + Newton steps, no IEEE division) and kept in
// shared memory; each block step then only applies its factors without
// normalisation (falling back to the normalised, protected solve when the
// result is not finite or too large) and runs the update with every load
// issued before its DFMAs.  Maxima and range checks use integer compares on
// the IEEE bit patterns.
//
// Per block step (block at local row q, size 1 or 2):
//   1. z = (T_qq - lambda I)^-1 rhs_q with pivots perturbed up to smin and a
//      power-of-two scale 2^sc <= 1 keeping |z| <= Omega (division
//      protection);
//   2. protect rows[0:q] -= T[0:q, q-block] z with nu + tau mu <= Omega
//      (tau = in-tile block norm, nu = running bound on the rows above,
//      recomputed exactly only when the bound asks for a scaling);
//   3. apply the update.
// All scalings are exact powers of two accumulated in the segment exponent
// e (y_true = y * 2^-e).
//
// Afterwards, for every tile r < s of each unit's column, the decisions of
// the update Y_r <- Y_r - T_rs X_s: a = min(e_r, e_s), protection q of
// (nu_r 2^(a-e_r), tau_rs, mu_s 2^(a-e_s)), new e_r = a + q,
// dy = a + q - e_r (scale of Y_r), dx = a + q - e_s (scale of X_s).
#include <algorithm>

#include "diag_big.cuh"
#include "diag_tile.cuh"

namespace evec {

// A programmatic launch (see grid_dependency_wait): the launch of the
// solve overlaps the end of the update kernel before it in the stream, and
// its prologue (the diagonal tile, the unit map and the block factors)
// reads only the input matrix and the plan.
template <typename... KArgs, typename... Args>
static void launch_programmatic(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                                size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// GR: lanes per real unit; GRC: the lane parameter of the complex units
// (Lanes<true, GRC>: 16 lanes per pair for GRC = 8, a whole warp for 16)
template <int W, bool GEN, bool RHS, int GR, int GRC = GR>
__global__ void __launch_bounds__(32 * W)
    k_diag_solve(int s, int nreal_ctas, const double *__restrict__ T, int64_t ldt, Plan P,
                 const double *__restrict__ tau, const double *__restrict__ blk_tau,
                 double *__restrict__ Y, int64_t ldy, int32_t *__restrict__ seg_e,
                 double *__restrict__ seg_nu, int32_t *__restrict__ seg_dx,
                 int32_t *__restrict__ seg_dy, Pencil pen, int decide) {
    extern __shared__ double smem[];
    if ((int)blockIdx.x < nreal_ctas)
        diag_tile<W, false, GEN, RHS, GR>(s, P.tile_real[s] + blockIdx.x * (Lanes<false, GR>::U * W),
                                          T, ldt, P, tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx,
                                          seg_dy, smem, pen, decide != 0);
    else
        diag_tile<W, true, GEN, RHS, GRC>(
            s, P.tile_cplx[s] + (blockIdx.x - nreal_ctas) * (Lanes<true, GRC>::U * W), T, ldt, P,
            tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx, seg_dy, smem, pen, decide != 0);
}

// Tiles of more than 64 rows: the sub-blocked solve (diag_big.cuh).
template <int W, bool GEN, bool RHS, int GR>
__global__ void __launch_bounds__(32 * W)
    k_diag_solve_big(int s, int nreal_ctas, const double *__restrict__ T, int64_t ldt, Plan P,
                     const double *__restrict__ tau, const double *__restrict__ blk_tau,
                     double *__restrict__ Y, int64_t ldy, int32_t *__restrict__ seg_e,
                     double *__restrict__ seg_nu, int32_t *__restrict__ seg_dx,
                     int32_t *__restrict__ seg_dy, Pencil pen, int decide) {
    extern __shared__ double smem[];
    if ((int)blockIdx.x < nreal_ctas)
        diag_tile_big<W, false, GEN, RHS, GR>(
            s, P.tile_real[s] + blockIdx.x * (Lanes<false, GR>::U * W), T, ldt, P, tau, blk_tau,
            Y, ldy, seg_e, seg_nu, seg_dx, seg_dy, smem, decide != 0, pen);
    else
        diag_tile_big<W, true, GEN, RHS, GR>(
            s, P.tile_cplx[s] + (blockIdx.x - nreal_ctas) * (Lanes<true, GR>::U * W), T, ldt, P,
            tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx, seg_dy, smem, decide != 0, pen);
}

template <int W, bool RHS, int GR = 8, bool GEN = false>
static int launch_big(int s, int ts, int nr, int nc, const double *T, int64_t ldt, const Plan &p,
                      const double *tau, const double *blk_tau, double *Y, int64_t ldy,
                      int32_t *seg_e, double *seg_nu, int32_t *seg_dx, int32_t *seg_dy,
                      cudaStream_t st, bool decide, int *sms, const Pencil &pen = Pencil()) {
    constexpr int ur = Lanes<false, GR>::U * W, uc = Lanes<true, GR>::U * W;
    const int rct = (nr + ur - 1) / ur;
    const int cct = (nc + uc - 1) / uc;
    if (rct + cct == 0) return 0;
    cudaFuncSetAttribute(k_diag_solve_big<W, GEN, RHS, GR>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_big_smem<W, GEN, GR>(kMaxTileBig));
    cudaFuncSetAttribute(k_diag_solve_big<W, GEN, RHS, GR>,
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    const size_t smem = diag_big_smem<W, GEN, GR>(ts);
    if (sms) {
        int per = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_diag_solve_big<W, GEN, RHS, GR>,
                                                          32 * W, smem) != cudaSuccess ||
            per < 1) {
            cudaGetLastError();
            per = 1;
        }
        *sms = (rct + cct + per - 1) / per;
        return 0;
    }
    launch_programmatic(k_diag_solve_big<W, GEN, RHS, GR>, (unsigned)(rct + cct), 32 * W, smem,
                        st, s, rct, T, ldt, p, tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx,
                        seg_dy, pen, decide ? 1 : 0);
    return 1;
}

// The decisions of step s for every active column and tile r < s (the
// last part of diag_tile, as its own launch when the diagonal solve ran
// with decide = 0): thread -> (column, tile row), consecutive threads on
// consecutive columns; a pair is handled at its real column.  Reads the
// segment exponent and maximum the solve left in seg_e / seg_nu of tile s.
template <bool RHS>
__global__ void __launch_bounds__(256)
    k_decide(int s, Plan P, const double *__restrict__ tau, int32_t *__restrict__ seg_e,
             double *__restrict__ seg_nu, int32_t *__restrict__ seg_dx,
             int32_t *__restrict__ seg_dy, int64_t c0) {
    const int64_t m = P.m, ncols = m - c0;
    const int64_t items = ncols * s;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < items;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + idx % ncols;
        const int r = (int)(idx / ncols);
        const int u = P.col_unit[c];
        const bool cplx = P.unit_lam[2 * u + 1] != 0.0;
        if (cplx && c != P.unit_col[u]) continue;
        const int64_t as = (int64_t)s * m + c, at = (int64_t)r * m + c;
        const int es = seg_e[as];
        const double mus = cplx ? fmax(seg_nu[as], seg_nu[as + 1]) : seg_nu[as];
        const bool ownu = !RHS && P.unit_tile[u] == s;   // fresh segments above the own block
        const int e_r = ownu ? es : seg_e[at];
        const double nur = ownu ? 0.0 : (cplx ? fmax(seg_nu[at], seg_nu[at + 1]) : seg_nu[at]);
        const int a = min(e_r, es);
        const int g2 = protect_update_scaled(nur, a - e_r, tau[(int64_t)r * P.ntiles + s], mus,
                                             a - es);
        const int ne = a + g2;
        seg_e[at] = ne;
        seg_dx[at] = ne - es;
        seg_dy[at] = ownu ? kFresh : ne - e_r;
        seg_nu[at] = 0.0;   // the update of this step writes the new maximum
        if (cplx) {
            seg_e[at + 1] = ne;
            seg_dx[at + 1] = ne - es;
            seg_dy[at + 1] = ownu ? kFresh : ne - e_r;
            seg_nu[at + 1] = 0.0;
        }
    }
}

void launch_decide(int s, const Plan &p, int64_t c0, const double *tau, int32_t *seg_e,
                   double *seg_nu, int32_t *seg_dx, int32_t *seg_dy, bool rhs, cudaStream_t st) {
    const int64_t items = (p.m - c0) * s;
    if (items <= 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>((items + 255) / 256, 4096);
    if (rhs)
        k_decide<true><<<grid, 256, 0, st>>>(s, p, tau, seg_e, seg_nu, seg_dx, seg_dy, c0);
    else
        k_decide<false><<<grid, 256, 0, st>>>(s, p, tau, seg_e, seg_nu, seg_dx, seg_dy, c0);
}

// dynamic shared memory of k_diag_solve<W, GEN, *, GR, GRC> for t rows
template <int W, bool GEN, int GR, int GRC>
static size_t diag_smem_mixed(int t) {
    return std::max(diag_smem_bytes<W, false, GEN, GR>(t), diag_smem_bytes<W, true, GEN, GRC>(t));
}

// CTAs of k_diag_solve<W, GEN, RHS, GR, GRC> resident on one SM for t rows
template <int W, bool GEN, bool RHS, int GR, int GRC>
static int diag_ctas_per_sm(int t) {
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_diag_solve<W, GEN, RHS, GR, GRC>,
                                                      32 * W,
                                                      diag_smem_mixed<W, GEN, GR, GRC>(t)) !=
            cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        per = 1;
    }
    return per;
}

template <int W, bool GEN, bool RHS, int GR = 8, int GRC = GR>
static int launch_w(int s, int ts, int nr, int nc, const double *T, int64_t ldt, const Plan &p,
                    const double *tau, const double *blk_tau, double *Y, int64_t ldy,
                    int32_t *seg_e, double *seg_nu, int32_t *seg_dx, int32_t *seg_dy,
                    const Pencil &pen, cudaStream_t st, bool decide, int *sms) {
    constexpr int ur = Lanes<false, GR>::U * W, uc = Lanes<true, GRC>::U * W;
    const int rct = (nr + ur - 1) / ur;
    const int cct = (nc + uc - 1) / uc;
    if (rct + cct == 0) return 0;
    cudaFuncSetAttribute(k_diag_solve<W, GEN, RHS, GR, GRC>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem_mixed<W, GEN, GR, GRC>(W == 4 ? 64 : kMaxTile));
    // two CTAs per SM at 8 lanes per real unit (about 82 KB each for 64-row
    // tiles; pencils: one), more with more lanes per unit
    cudaFuncSetAttribute(k_diag_solve<W, GEN, RHS, GR, GRC>,
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    const size_t smem = diag_smem_mixed<W, GEN, GR, GRC>(ts);
    if (sms) {   // SMs the launch occupies in one wave (planning only: no launch)
        const int per = diag_ctas_per_sm<W, GEN, RHS, GR, GRC>(ts);
        *sms = (rct + cct + per - 1) / per;
        return 0;
    }
    launch_programmatic(k_diag_solve<W, GEN, RHS, GR, GRC>, (unsigned)(rct + cct), 32 * W, smem,
                        st, s, rct, T, ldt, p, tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx,
                        seg_dy, pen, decide ? 1 : 0);
    return 1;
}

// Lanes per real unit for a step with nr real and nc complex active units.
// A unit's chain is latency-bound: per block step its lanes issue the
// update of the rows above as ceil(q / G) dependent-issue DFMAs, so more
// lanes per unit shorten every step while the sub-partitions have warps to
// spare; with many units the FP64 issue slots fill up and the solve work
// that every lane of a unit repeats makes wide units the slower choice.
// Largest GR with about 2.5 warps per SM sub-partition at most.
static int sm_count() {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            nsm = v;
        else
            nsm = 148;
    }
    return nsm;
}

static int pick_lanes(int nr, int nc) {
    const int nsm = sm_count();
    const double cap = 2.5 * 4.0 * nsm;
    for (int gr : {32, 16}) {
        const double warps = nr * gr / 32.0 + nc * std::min(2 * gr, 32) / 32.0;
        if (warps <= cap) return gr;
    }
    return 8;
}

// Returns the number of kernels launched (0 when no column is active).
// pen: the pencil's second matrix (tiles of at most 64 rows), or null.
// rhs: solve from the right-hand side already in Y (standard problem).
int launch_diag_solve(int s, const double *T, int64_t ldt, const Plan &p,
                      const int32_t *tile_start_h, const int32_t *tile_real_h,
                      const int32_t *tile_cplx_h, const double *tau, const double *blk_tau,
                      double *Y, int64_t ldy, int32_t *seg_e, double *seg_nu, int32_t *seg_dx,
                      int32_t *seg_dy, cudaStream_t st, const Pencil *pen, bool rhs,
                      bool decide, int *sms) {
    const int ts = tile_start_h[s + 1] - tile_start_h[s];
    const int nr = p.nreal - tile_real_h[s];
    const int nc = p.ncplx - tile_cplx_h[s];
    if (pen && ts > 64)   // pencil tiles above 64 rows: the sub-blocked solve
        return launch_big<4, false, 8, true>(s, ts, nr, nc, T, ldt, p, tau, blk_tau, Y, ldy,
                                             seg_e, seg_nu, seg_dx, seg_dy, st, decide, sms, *pen);
    if (pen)
        return launch_w<4, true, false>(s, ts, nr, nc, T, ldt, p, tau, blk_tau, Y, ldy, seg_e,
                                        seg_nu, seg_dx, seg_dy, *pen, st, decide, sms);
    const int gr = pick_lanes(nr, nc);
    // tiles above 64 rows: the sub-blocked solve, four warps per CTA
    if (ts > 64) {
#define EVEC_BIG_LAUNCH(R, G_)                                                                   \
    return launch_big<4, R, G_>(s, ts, nr, nc, T, ldt, p, tau, blk_tau, Y, ldy, seg_e, seg_nu,     \
                                seg_dx, seg_dy, st, decide, sms)
        if (rhs) {
            if (gr == 32) EVEC_BIG_LAUNCH(true, 32);
            if (gr == 16) EVEC_BIG_LAUNCH(true, 16);
            EVEC_BIG_LAUNCH(true, 8);
        }
        if (gr == 32) EVEC_BIG_LAUNCH(false, 32);
        if (gr == 16) EVEC_BIG_LAUNCH(false, 16);
        EVEC_BIG_LAUNCH(false, 8);
#undef EVEC_BIG_LAUNCH
    }
#define EVEC_DIAG_LAUNCH(R, G_, GC_)                                                             \
    return launch_w<4, false, R, G_, GC_>(s, ts, nr, nc, T, ldt, p, tau, blk_tau, Y, ldy, seg_e,  \
                                          seg_nu, seg_dx, seg_dy, Pencil(), st, decide, sms)
    // With complex pairs in the step, a pair's chain (complex arithmetic,
    // twice the FP64 instructions of a real column per block step) is the
    // longest one of the launch, and the real units are given 8 lanes: their
    // chain stays shorter, and their warps leave the sub-partitions' FP64
    // issue slots to the pairs.  The pairs take a whole warp each when the
    // launch still fits in one wave of resident CTAs, else 16 lanes.
    if (nc > 0) {
        const int nsm = sm_count();
        const int wide = (nr + 15) / 16 + (nc + 3) / 4;   // CTAs with a warp per pair
        const bool fits =
            wide <= nsm * (rhs ? diag_ctas_per_sm<4, false, true, 8, 16>(ts)
                               : diag_ctas_per_sm<4, false, false, 8, 16>(ts));
        if (rhs) {
            if (fits) EVEC_DIAG_LAUNCH(true, 8, 16);
            EVEC_DIAG_LAUNCH(true, 8, 8);
        }
        if (fits) EVEC_DIAG_LAUNCH(false, 8, 16);
        EVEC_DIAG_LAUNCH(false, 8, 8);
    }
    if (rhs) {
        if (gr == 32) EVEC_DIAG_LAUNCH(true, 32, 32);
        if (gr == 16) EVEC_DIAG_LAUNCH(true, 16, 16);
        EVEC_DIAG_LAUNCH(true, 8, 8);
    }
    if (gr == 32) EVEC_DIAG_LAUNCH(false, 32, 32);
    if (gr == 16) EVEC_DIAG_LAUNCH(false, 16, 16);
    EVEC_DIAG_LAUNCH(false, 8, 8);
#undef EVEC_DIAG_LAUNCH
}

}  // namespace evec
