// k_diag_solve.cu -- robust shifted solves on one diagonal tile (Eq. evec_solve
// restricted to the rows of tile s), then the consolidation/protection
// decisions for every tile above it (Sec. 3.4, the preprocessing step of the
// update Z <- Y - T X).
//
// One warp per unit (a real eigenvalue, or a complex pair solved as one
// complex column).  T_ss sits in shared memory and is shared by the CTA's
// warps; the unit's tile segment lives in a per-warp shared buffer.  Every
// unit runs its own chain of block steps from the bottom of the tile to the
// top; within a step the rows above the block are updated by the 32 lanes.
//
// Per block step (block at local row q, size 1 or 2):
//   1. solve (T_qq - lambda I) z = rhs_q, 1x1 or 2x2, real or complex, with
//      pivots perturbed up to smin and a power-of-two scale 2^sc <= 1 chosen
//      so |z| <= Omega (the division protection);
//   2. protect the update rows[0:q] -= T[0:q, q-block] z with the bound
//      nu + tau mu <= Omega (tau = blk_tau, nu = running bound on the rows,
//      recomputed exactly only when the bound asks for a scaling);
//   3. apply the update.
// All scalings are exact powers of two and accumulate in the segment's
// exponent e (y_true = y * 2^-e).
//
// Afterwards, for every tile r < s of the unit's column, the decisions of
// the update Y_r <- Y_r - T_rs X_s are taken here: common exponent
// a = min(e_r, e_s), protection q of (nu_r 2^(a-e_r), tau_rs, mu_s 2^(a-e_s)),
// new e_r = a + q, and the two scale exponents dy = a + q - e_r (for Y_r) and
// dx = a + q - e_s (for X_s), consumed by the update kernel.
#include "evec_internal.cuh"

namespace evec {

namespace {

struct Cx {
    double re, im;
};

__device__ __forceinline__ double abs1(Cx a) { return fabs(a.re) + fabs(a.im); }
__device__ __forceinline__ double absmax(Cx a) { return fmax(fabs(a.re), fabs(a.im)); }
__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ Cx csub(Cx a, Cx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cx cscale(Cx a, int k) { return {scale2(a.re, k), scale2(a.im, k)}; }

// a / b by Smith's method (no intermediate above ~2 max|a| / max|b|).
__device__ __forceinline__ Cx cdiv(Cx a, Cx b) {
    if (fabs(b.re) >= fabs(b.im)) {
        double t = b.im / b.re, d = b.re + b.im * t;
        return {(a.re + a.im * t) / d, (a.im - a.re * t) / d};
    }
    double t = b.re / b.im, d = b.im + b.re * t;
    return {(a.re * t + a.im) / d, (a.im * t - a.re) / d};
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Solve the bs x bs shifted system at local row q; returns sc <= 0 and
// z with M z = 2^sc rhs, |z| <= Omega.  Ts: tile in shared memory, ld ts.
__device__ int small_solve(int bs, const double *Ts, int ts, int q, double lr, double li,
                           double smin, Cx r0, Cx r1, Cx &z0, Cx &z1) {
    z1 = {0.0, 0.0};
    if (bs == 1 && li == 0.0) {
        // real 1x1: the common case, decided directly on the pivot
        double piv = Ts[q + q * ts] - lr;
        if (fabs(piv) < smin) piv = smin;
        const double rn = fabs(r0.re);
        if (rn == 0.0) { z0 = {0.0, 0.0}; return 0; }
        int sc = 0;
        double rr = r0.re;
        if (fabs(piv) < 1.0 && rn > kOmega * fabs(piv)) {
            sc = ilog2_abs(kOmega * piv) - ilog2_abs(rn) - 1;
            rr = scale2(rr, sc);
        }
        z0 = {rr / piv, 0.0};
        return sc;
    }
    // general case: normalise the right-hand side, solve with complete
    // pivoting, then fit the scale to the computed solution
    double rn = fmax(absmax(r0), bs == 2 ? absmax(r1) : 0.0);
    if (rn == 0.0) { z0 = {0.0, 0.0}; return 0; }
    const int kr = ilog2_abs(rn) + 1;
    Cx c0 = cscale(r0, -kr), c1 = cscale(r1, -kr);
    Cx h0, h1 = {0.0, 0.0};
    if (bs == 1) {
        Cx piv = {Ts[q + q * ts] - lr, -li};
        if (abs1(piv) < smin) piv = {smin, 0.0};
        h0 = cdiv(c0, piv);
    } else {
        Cx M[2][2];
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++) {
                double t = Ts[(q + a) + (q + b) * ts];
                M[a][b] = (a == b) ? Cx{t - lr, -li} : Cx{t, 0.0};
            }
        int pr = 0, pc = 0;
        double best = -1.0;
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 2; b++)
                if (abs1(M[a][b]) > best) { best = abs1(M[a][b]); pr = a; pc = b; }
        Cx a11 = M[pr][pc], a12 = M[pr][1 - pc];
        Cx a21 = M[1 - pr][pc], a22 = M[1 - pr][1 - pc];
        Cx d1 = pr == 0 ? c0 : c1, d2 = pr == 0 ? c1 : c0;
        if (abs1(a11) < smin) a11 = {smin, 0.0};
        Cx l = cdiv(a21, a11);
        Cx u = csub(a22, cmul(l, a12));
        if (abs1(u) < smin) u = {smin, 0.0};
        Cx w2 = cdiv(csub(d2, cmul(l, d1)), u);
        Cx w1 = csub(cdiv(d1, a11), cmul(cdiv(a12, a11), w2));
        // w1 belongs to column pc, w2 to column 1 - pc
        h0 = pc == 0 ? w1 : w2;
        h1 = pc == 0 ? w2 : w1;
    }
    double hn = fmax(absmax(h0), absmax(h1));
    if (hn == 0.0) { z0 = {0.0, 0.0}; z1 = {0.0, 0.0}; return 0; }
    int sc = kOmegaExp - ilog2_abs(hn) - 1 - kr;
    if (sc > 0) sc = 0;
    z0 = cscale(h0, kr + sc);
    z1 = cscale(h1, kr + sc);
    return sc;
}

}  // namespace

template <int NWARP>
__global__ void __launch_bounds__(NWARP * 32)
    k_diag_solve(int s, const double *__restrict__ T, int64_t ldt, Plan P,
                 const double *__restrict__ tau, const double *__restrict__ blk_tau,
                 double *__restrict__ Y, int64_t ldy, int32_t *__restrict__ seg_e,
                 double *__restrict__ seg_nu, int32_t *__restrict__ seg_dx,
                 int32_t *__restrict__ seg_dy) {
    extern __shared__ double smem[];
    const int t0 = P.tile_start[s];
    const int ts = P.tile_start[s + 1] - t0;
    double *Ts = smem;                                   // ts x ts, ld ts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *yr = smem + ts * ts + warp * 2 * kMaxTile;
    double *yi = yr + kMaxTile;

    for (int idx = threadIdx.x; idx < ts * ts; idx += NWARP * 32) {
        const int i = idx % ts, j = idx / ts;
        Ts[idx] = (i <= j + 1) ? T[(t0 + i) + (int64_t)(t0 + j) * ldt] : 0.0;
    }
    __syncthreads();

    const int u = P.tile_unit[s] + blockIdx.x * NWARP + warp;
    if (u >= P.nunits) return;

    const int64_t m = P.m;
    const int col = P.unit_col[u];
    const int kown = P.unit_blk[u];
    const bool own = P.unit_tile[u] == s;
    const double lr = P.unit_lam[2 * u], li = P.unit_lam[2 * u + 1];
    const bool cplx = li != 0.0;
    double smin = kUlp * (fabs(lr) + fabs(li));
    smin = fmax(smin, kSafeMin * ((double)P.n / kUlp));
    const int kb0 = P.tile_blk[s], kb1 = P.tile_blk[s + 1];

    int e = 0;
    double nu = 0.0;      // running upper bound on |rows above the current block|
    int kfirst;           // first block to solve, going up

    // scale every row of the segment (and the caller's z) by 2^g
    auto scale_all = [&](int g) {
        for (int i = lane; i < ts; i += 32) {
            yr[i] = scale2(yr[i], g);
            yi[i] = scale2(yi[i], g);
        }
    };

    // protected update of rows [0, q) from block k whose solution is z
    auto update_from = [&](int k, int q, int bs, Cx z0, Cx z1) {
        double mu = fmax(absmax(z0), absmax(z1));
        const double tq = blk_tau[k];
        int g = protect_update(nu, tq, mu);
        if (g != 0) {
            // the bound asks for a scaling: recompute the rows' true maximum
            double loc = 0.0;
            for (int i = lane; i < q; i += 32) loc = fmax(loc, fmax(fabs(yr[i]), fabs(yi[i])));
            nu = warp_max(loc);
            g = protect_update(nu, tq, mu);
            if (g != 0) {
                __syncwarp();
                scale_all(g);
                z0 = cscale(z0, g);
                z1 = cscale(z1, g);
                mu = scale2(mu, g);
                nu = scale2(nu, g);
                e += g;
            }
        }
        __syncwarp();
        const double *c0 = Ts + q * ts;
        const double *c1 = Ts + (q + 1) * ts;
        if (bs == 1) {
            for (int i = lane; i < q; i += 32) {
                const double t = c0[i];
                yr[i] = fma(-t, z0.re, yr[i]);
                yi[i] = fma(-t, z0.im, yi[i]);
            }
        } else {
            for (int i = lane; i < q; i += 32) {
                const double ta = c0[i], tb = c1[i];
                yr[i] = fma(-tb, z1.re, fma(-ta, z0.re, yr[i]));
                yi[i] = fma(-tb, z1.im, fma(-ta, z0.im, yi[i]));
            }
        }
        nu = nu + tq * mu;
        __syncwarp();
    };

    if (own) {
        for (int i = lane; i < ts; i += 32) { yr[i] = 0.0; yi[i] = 0.0; }
        __syncwarp();
        const int q = P.blk_start[kown] - t0;
        const int bs = P.blk_size[kown];
        const double *o = P.unit_own + 4 * u;
        Cx z0 = {o[0], o[2]}, z1 = {o[1], o[3]};
        if (lane == 0) {
            yr[q] = z0.re; yi[q] = z0.im;
            if (bs == 2) { yr[q + 1] = z1.re; yi[q + 1] = z1.im; }
        }
        __syncwarp();
        if (bs == 1) z1 = {0.0, 0.0};
        if (q > 0) update_from(kown, q, bs, z0, z1);
        kfirst = kown - 1;
    } else {
        const double *gr = Y + (int64_t)col * ldy + t0;
        const double *gi = Y + (int64_t)(col + 1) * ldy + t0;
        double loc = 0.0;
        for (int i = lane; i < ts; i += 32) {
            const double a = gr[i];
            const double b = cplx ? gi[i] : 0.0;
            yr[i] = a;
            yi[i] = b;
            loc = fmax(loc, fmax(fabs(a), fabs(b)));
        }
        nu = warp_max(loc);
        e = seg_e[(int64_t)s * m + col];
        kfirst = kb1 - 1;
        __syncwarp();
    }

    for (int k = kfirst; k >= kb0; k--) {
        const int q = P.blk_start[k] - t0;
        const int bs = P.blk_size[k];
        Cx r0 = {yr[q], yi[q]};
        Cx r1 = bs == 2 ? Cx{yr[q + 1], yi[q + 1]} : Cx{0.0, 0.0};
        Cx z0, z1;
        const int sc = small_solve(bs, Ts, ts, q, lr, li, smin, r0, r1, z0, z1);
        __syncwarp();
        if (sc != 0) {
            scale_all(sc);
            nu = scale2(nu, sc);
            e += sc;
            __syncwarp();
        }
        if (lane == 0) {
            yr[q] = z0.re; yi[q] = z0.im;
            if (bs == 2) { yr[q + 1] = z1.re; yi[q + 1] = z1.im; }
        }
        __syncwarp();
        if (q > 0) update_from(k, q, bs, z0, z1);
    }

    // write the solved segment back, with its exponent and column maxima
    double mr = 0.0, mi = 0.0;
    {
        double *gr = Y + (int64_t)col * ldy + t0;
        double *gi = Y + (int64_t)(col + 1) * ldy + t0;
        for (int i = lane; i < ts; i += 32) {
            gr[i] = yr[i];
            mr = fmax(mr, fabs(yr[i]));
            if (cplx) {
                gi[i] = yi[i];
                mi = fmax(mi, fabs(yi[i]));
            }
        }
    }
    mr = warp_max(mr);
    mi = warp_max(mi);
    if (lane == 0) {
        seg_e[(int64_t)s * m + col] = e;
        seg_nu[(int64_t)s * m + col] = mr;
        if (cplx) {
            seg_e[(int64_t)s * m + col + 1] = e;
            seg_nu[(int64_t)s * m + col + 1] = mi;
        }
    }
    const double mu_s = fmax(mr, mi);

    // consolidation + protection decisions for the tiles above (Sec. 3.4)
    for (int r = lane; r < s; r += 32) {
        const int64_t at = (int64_t)r * m + col;
        int er;
        double nur;
        if (own) {
            er = e;
            nur = 0.0;
        } else {
            er = seg_e[at];
            nur = seg_nu[at];
            if (cplx) nur = fmax(nur, seg_nu[at + 1]);
        }
        const int a = min(er, e);
        const double nup = scale2(nur, a - er);
        const double mup = scale2(mu_s, a - e);
        const int g = protect_update(nup, tau[(int64_t)r * P.ntiles + s], mup);
        const int ne = a + g;
        seg_e[at] = ne;
        seg_dx[at] = ne - e;
        seg_dy[at] = own ? kFresh : ne - er;
        if (cplx) {
            seg_e[at + 1] = ne;
            seg_dx[at + 1] = ne - e;
            seg_dy[at + 1] = own ? kFresh : ne - er;
        }
    }
}

constexpr int kSolveWarps = 16;

void launch_diag_solve(int s, const double *T, int64_t ldt, const Plan &p,
                       const int32_t *tile_start_h, const int32_t *tile_unit_h,
                       const double *tau, const double *blk_tau, double *Y, int64_t ldy,
                       int32_t *seg_e, double *seg_nu, int32_t *seg_dx, int32_t *seg_dy,
                       cudaStream_t st) {
    const int ts = tile_start_h[s + 1] - tile_start_h[s];
    const int units = p.nunits - tile_unit_h[s];
    if (units <= 0) return;
    const int blocks = (units + kSolveWarps - 1) / kSolveWarps;
    const size_t shm = sizeof(double) * ((size_t)ts * ts + (size_t)kSolveWarps * 2 * kMaxTile);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_diag_solve<kSolveWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * ((size_t)kMaxTile * kMaxTile +
                                                     (size_t)kSolveWarps * 2 * kMaxTile)));
        attr_set = true;
    }
    k_diag_solve<kSolveWarps><<<blocks, kSolveWarps * 32, shm, st>>>(
        s, T, ldt, p, tau, blk_tau, Y, ldy, seg_e, seg_nu, seg_dx, seg_dy);
}

}  // namespace evec
