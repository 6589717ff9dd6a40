// diag_tile.cuh -- the robust diagonal-tile solve of one tile for a chunk of
// units, as a device function: used by the per-step kernel (k_diag_solve.cu)
// and by the batched persistent kernel (k_batched.cu).  The design notes are
// at the top of k_diag_solve.cu.
#pragma once

#include "evec_internal.cuh"

namespace evec {

namespace {

// GR lanes per real unit (8, 16 or 32), twice that (at most a warp) per
// complex pair
template <bool C, int GR = 8>
struct Lanes {
    static constexpr int G = C ? (2 * GR < 32 ? 2 * GR : 32) : GR;   // lanes per unit
    static constexpr int U = 32 / G;                                   // units per warp
};

struct Cx {
    double re, im;
};

template <bool C>
__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
    if (!C) return {a.re * b.re, 0.0};
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ Cx csub(Cx a, Cx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cx cscale(Cx a, int k) { return {scale2(a.re, k), scale2(a.im, k)}; }
__device__ __forceinline__ long long cbits(Cx a) { return max(abs_bits(a.re), abs_bits(a.im)); }

// 1 / a, a != 0: (re - i im) / (re^2 + im^2) after an exact power-of-two
// normalisation of a.
__device__ __forceinline__ Cx crcp(Cx a) {
    if (a.im == 0.0) return {rcp_fast(a.re), 0.0};
    const int k = ilog2_abs(__longlong_as_double(cbits(a)));
    const double ar = scale2(a.re, -k), ai = scale2(a.im, -k);
    const double id = rcp_fast(fma(ar, ar, ai * ai));
    return {scale2(ar * id, -k), scale2(-ai * id, -k)};
}

// Factors of the shifted block system M = T_qq - lambda I (complete
// pivoting for 2x2, pivots below smin replaced by smin).
struct Fac {
    Cx ia, l, g, iu;
    int pr, pc;
};

// |a|_max key for pivot choice: high word of the larger component (the order
// of non-negative doubles restricted to their high words; ties arbitrary)
__device__ __forceinline__ int pkey(Cx a) {
    return max(__double2hiint(a.re) & 0x7fffffff, __double2hiint(a.im) & 0x7fffffff);
}
// "below smin" on exponent fields: |a|_max < 2^(field(smin) - 1023) <= smin
__device__ __forceinline__ bool tiny(Cx a, int fsmin) {
    return max(efield(a.re), efield(a.im)) < fsmin;
}

// LU with complete pivoting of the 1x1 / 2x2 block system M (pivots below
// smin replaced by smin)
template <bool C>
__device__ Fac factor_matrix(int bs, Cx (&M)[2][2], double smin) {
    Fac F;
    F.pr = F.pc = 0;
    F.l = F.g = F.iu = {0.0, 0.0};
    const int fsmin = efield(smin);
    if (bs == 1) {
        Cx p = M[0][0];
        if (tiny(p, fsmin)) p = {smin, 0.0};
        F.ia = crcp(p);
        return F;
    }
    int best = -1;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int v = pkey(M[a][b]);
            if (v > best) { best = v; F.pr = a; F.pc = b; }
        }
    Cx a11 = M[F.pr][F.pc];
    const Cx a12 = M[F.pr][1 - F.pc], a21 = M[1 - F.pr][F.pc], a22 = M[1 - F.pr][1 - F.pc];
    if (tiny(a11, fsmin)) a11 = {smin, 0.0};
    F.ia = crcp(a11);
    F.l = cmul<C>(a21, F.ia);
    F.g = cmul<C>(a12, F.ia);
    Cx u = csub(a22, cmul<C>(F.l, a12));
    if (tiny(u, fsmin)) u = {smin, 0.0};
    F.iu = crcp(u);
    return F;
}

// The diagonal tile of diag_tile is kept in shared memory packed by
// columns: column j holds rows 0 .. j + 1 (the upper part and the first
// subdiagonal, all a quasi-triangular tile has) from pk_col(j) on, about
// half of a square ts x ts array.
__host__ __device__ constexpr int pk_col(int j) { return j * (j + 3) / 2; }
__host__ __device__ constexpr int pk_size(int t) { return t * (t + 3) / 2; }

// entry (i, j) of a tile: packed (PK, i <= j + 1) or square with ld
template <bool PK>
__device__ __forceinline__ double tile_at(const double *A, int ld, int i, int j) {
    return PK ? A[pk_col(j) + i] : A[i + j * ld];
}

// factors of T_qq - lambda I
template <bool C, bool PK = false>
__device__ Fac factor(int bs, const double *Ts, int ts, int q, double lr, double li, double smin) {
    Cx M[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            if (a >= bs || b >= bs) { M[a][b] = {0.0, 0.0}; continue; }
            const double t = tile_at<PK>(Ts, ts, q + a, q + b);
            M[a][b] = (a == b) ? Cx{t - lr, C ? -li : 0.0} : Cx{t, 0.0};
        }
    return factor_matrix<C>(bs, M, smin);
}

// factors of beta S_qq - alpha T_qq (pencil; T upper triangular)
template <bool C, bool PK = false>
__device__ Fac factor_pencil(int bs, const double *Ss, const double *Tt, int ts, int q, double ar,
                             double ai, double be, double smin) {
    Cx M[2][2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
            if (a >= bs || b >= bs) { M[a][b] = {0.0, 0.0}; continue; }
            const double sv = tile_at<PK>(Ss, ts, q + a, q + b);
            const double tv = b >= a ? tile_at<PK>(Tt, ts, q + a, q + b) : 0.0;
            M[a][b] = {be * sv - ar * tv, C ? -ai * tv : 0.0};
        }
    return factor_matrix<C>(bs, M, smin);
}

// The lanes of one unit: the lane group's mask (G lanes from a multiple of G)
template <int G>
__device__ __forceinline__ unsigned unit_mask() {
    if constexpr (G >= 32) return 0xffffffffu;
    else return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

// A complex value whose real part is formed on the even lanes of a unit and
// its imaginary part on the odd ones: each lane holds its own part in `mine`;
// the pair of lanes (g, g ^ 1) swaps them.
__device__ __forceinline__ Cx cx_join(double mine, bool odd, unsigned mask) {
    const double other = __shfl_xor_sync(mask, mine, 1);
    return odd ? Cx{other, mine} : Cx{mine, other};
}

// Complex case of apply: the same FP64 expressions, component by component,
// as the form below, but each lane evaluates only its own component (even
// lanes the real parts, odd lanes the imaginary ones) and the partner lane
// supplies the other.  On B300 an FP64 warp instruction costs its
// sub-partition 64 cycles whatever its active lanes, so this halves the
// FP64 instructions of a complex pair's small solves (1x1: 2 instead of 4,
// 2x2: 8 instead of 16) on the critical chain; the results are
// bit-identical (the operand selections and negations are exact).
__device__ __forceinline__ void apply_split(const Fac &F, int bs, Cx r0, Cx r1, Cx &z0, Cx &z1,
                                            bool odd, unsigned mask) {
    if (bs == 1) {
        // z0 = r0 ia: re = fma(r.re, ia.re, -r.im ia.im), im = fma(r.re, ia.im, r.im ia.re)
        const double p = r0.im * (odd ? F.ia.re : F.ia.im);
        const double v = fma(r0.re, odd ? F.ia.im : F.ia.re, odd ? p : -p);
        z0 = cx_join(v, odd, mask);
        z1 = {0.0, 0.0};
        return;
    }
    const Cx d1 = F.pr == 0 ? r0 : r1, d2 = F.pr == 0 ? r1 : r0;
    // t = d2 - l d1:
    //   re = fma(-l.re, d1.re, fma(l.im, d1.im, d2.re))
    //   im = fma(-l.re, d1.im, fma(-l.im, d1.re, d2.im))
    const double ti = fma(odd ? -F.l.im : F.l.im, odd ? d1.re : d1.im, odd ? d2.im : d2.re);
    const Cx t = cx_join(fma(-F.l.re, odd ? d1.im : d1.re, ti), odd, mask);
    // w2 = t iu, as cmul
    const double q = t.im * (odd ? F.iu.re : F.iu.im);
    const Cx w2 = cx_join(fma(t.re, odd ? F.iu.im : F.iu.re, odd ? q : -q), odd, mask);
    // w1 = d1 ia - g w2:
    //   re = fma(d1.re, ia.re, fma(-d1.im, ia.im, fma(-g.re, w2.re, g.im w2.im)))
    //   im = fma(d1.re, ia.im, fma(d1.im, ia.re, fma(-g.re, w2.im, -g.im w2.re)))
    const double m = (odd ? -F.g.im : F.g.im) * (odd ? w2.re : w2.im);
    const double a1 = fma(-F.g.re, odd ? w2.im : w2.re, m);
    const double a2 = fma(odd ? d1.im : -d1.im, odd ? F.ia.re : F.ia.im, a1);
    const Cx w1 = cx_join(fma(d1.re, odd ? F.ia.im : F.ia.re, a2), odd, mask);
    z0 = F.pc == 0 ? w1 : w2;
    z1 = F.pc == 0 ? w2 : w1;
}

template <bool C>
__device__ __forceinline__ void apply(const Fac &F, int bs, Cx r0, Cx r1, Cx &z0, Cx &z1) {
    if (bs == 1) {
        z0 = cmul<C>(r0, F.ia);
        z1 = {0.0, 0.0};
        return;
    }
    const Cx d1 = F.pr == 0 ? r0 : r1, d2 = F.pr == 0 ? r1 : r0;
    Cx t;   // d2 - l d1, fused
    if (C) {
        t.re = fma(-F.l.re, d1.re, fma(F.l.im, d1.im, d2.re));
        t.im = fma(-F.l.re, d1.im, fma(-F.l.im, d1.re, d2.im));
    } else {
        t = {fma(-F.l.re, d1.re, d2.re), 0.0};
    }
    const Cx w2 = cmul<C>(t, F.iu);
    Cx w1;  // d1 ia - g w2, fused
    if (C) {
        w1.re = fma(d1.re, F.ia.re, fma(-d1.im, F.ia.im, fma(-F.g.re, w2.re, F.g.im * w2.im)));
        w1.im = fma(d1.re, F.ia.im, fma(d1.im, F.ia.re, fma(-F.g.re, w2.im, -F.g.im * w2.re)));
    } else {
        w1 = {fma(d1.re, F.ia.re, -F.g.re * w2.re), 0.0};
    }
    z0 = F.pc == 0 ? w1 : w2;
    z1 = F.pc == 0 ? w2 : w1;
}

// Solve with the division protection: the unnormalised application is
// exact up to rounding whenever its result is finite and <= Omega (an
// intermediate overflow always leaves an Inf or NaN in the result);
// otherwise normalise the right-hand side, apply again and fit sc <= 0.
// Complex units (C): every lane of the unit's group (mask) calls this
// together, with odd = its lane parity within the group.
template <bool C>
__device__ __forceinline__ void apply_any(const Fac &F, int bs, Cx r0, Cx r1, Cx &z0, Cx &z1,
                                         bool odd, unsigned mask) {
    if (C) apply_split(F, bs, r0, r1, z0, z1, odd, mask);
    else apply<C>(F, bs, r0, r1, z0, z1);
}

template <bool C>
__device__ __forceinline__ int solve(const Fac &F, int bs, Cx r0, Cx r1, Cx &z0, Cx &z1,
                                     bool odd, unsigned mask) {
    apply_any<C>(F, bs, r0, r1, z0, z1, odd, mask);
    // |z| < 2^1020 (and finite) on the exponent fields alone
    const int fz = max(max(efield(z0.re), efield(z0.im)), max(efield(z1.re), efield(z1.im)));
    if (fz <= 2042) return 0;
    const long long rb = max(cbits(r0), cbits(r1));
    if (rb == 0) { z0 = {0.0, 0.0}; z1 = {0.0, 0.0}; return 0; }
    const int kr = ilog2_abs(__longlong_as_double(rb)) + 1;
    Cx h0, h1;
    apply_any<C>(F, bs, cscale(r0, -kr), cscale(r1, -kr), h0, h1, odd, mask);
    const long long hb = max(cbits(h0), cbits(h1));
    if (hb == 0) { z0 = {0.0, 0.0}; z1 = {0.0, 0.0}; return 0; }
    int sc = kOmegaExp - ilog2_abs(__longlong_as_double(hb)) - 1 - kr;
    if (sc > 0) sc = 0;
    z0 = cscale(h0, kr + sc);
    z1 = cscale(h1, kr + sc);
    return sc;
}

template <int G>
__device__ __forceinline__ long long group_max_bits(long long v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc));
}

// rows [0, q) of one unit -= T[0:q, q-block] z: the lane's rows g, g + G, ...
// from the highest down (the rows of the next block to solve come first),
// with a trip count uniform across the warp, two rows per step (loads first)
template <bool C, int BS, int G>
__device__ __forceinline__ void update_rows(double *myr, double *myi, const double *c0,
                                            const double *c1, int q, int g, Cx z0, Cx z1,
                                            int ys) {
    const int n = (q + G - 1) / G;
    int j = n - 1;
    for (; j >= 1; j -= 2) {
        const int i0 = g + G * j, i1 = i0 - G;
        const bool ok0 = i0 < q;            // only the highest row can be beyond q
        const double a0 = ok0 ? myr[i0 * ys] : 0.0, a1 = myr[i1 * ys];
        const double b0 = (C && ok0) ? myi[i0 * ys] : 0.0, b1 = C ? myi[i1 * ys] : 0.0;
        const double t0 = ok0 ? c0[i0] : 0.0, t1 = c0[i1];
        const double u0 = (BS == 2 && ok0) ? c1[i0] : 0.0, u1 = BS == 2 ? c1[i1] : 0.0;
        double v0 = fma(-t0, z0.re, a0), v1 = fma(-t1, z0.re, a1);
        if (BS == 2) { v0 = fma(-u0, z1.re, v0); v1 = fma(-u1, z1.re, v1); }
        if (ok0) myr[i0 * ys] = v0;
        myr[i1 * ys] = v1;
        if (C) {
            double w0 = fma(-t0, z0.im, b0), w1 = fma(-t1, z0.im, b1);
            if (BS == 2) { w0 = fma(-u0, z1.im, w0); w1 = fma(-u1, z1.im, w1); }
            if (ok0) myi[i0 * ys] = w0;
            myi[i1 * ys] = w1;
        }
    }
    if (j == 0 && g < q) {
        const int i = g;
        double v = fma(-c0[i], z0.re, myr[i * ys]);
        if (BS == 2) v = fma(-c1[i], z1.re, v);
        myr[i * ys] = v;
        if (C) {
            double w = fma(-c0[i], z0.im, myi[i * ys]);
            if (BS == 2) w = fma(-c1[i], z1.im, w);
            myi[i * ys] = w;
        }
    }
}

// The whole kernel for one kind of unit (real or complex) and W warps.
// pencils: rows [0, q) -= S[0:q, block] (beta z) - T[0:q, block] (alpha z),
// with zb = beta z and wz = alpha z precomputed per block
template <bool C, int BS, int G>
__device__ __forceinline__ void update_rows_pencil(double *myr, double *myi, const double *s0,
                                                   const double *s1, const double *t0c,
                                                   const double *t1c, int q, int g, Cx zb0, Cx zb1,
                                                   Cx wz0, Cx wz1, int ys) {
    const int n = (q + G - 1) / G;
    for (int j = n - 1; j >= 0; j--) {   // highest rows first
        const int i = g + G * j;
        if (i >= q) continue;
        const double a = myr[i * ys];
        const double b = C ? myi[i * ys] : 0.0;
        const double sa = s0[i], ta = t0c[i];
        const double sb = BS == 2 ? s1[i] : 0.0, tb = BS == 2 ? t1c[i] : 0.0;
        double v = fma(ta, wz0.re, fma(-sa, zb0.re, a));
        if (BS == 2) v = fma(tb, wz1.re, fma(-sb, zb1.re, v));
        myr[i * ys] = v;
        if (C) {
            double w = fma(ta, wz0.im, fma(-sa, zb0.im, b));
            if (BS == 2) w = fma(tb, wz1.im, fma(-sb, zb1.im, w));
            myi[i * ys] = w;
        }
    }
}

// RHS: the segments start from a given right-hand side instead of the
// eigenvector's own block: every unit (own tile included) loads its rows of
// Y with exponents seg_e and maxima seg_nu, the own block is fixed at zero,
// and no segment is fresh (the correction solve of the residual sweep).
template <int W, bool C, bool GEN = false, bool RHS = false, int GR = 8>
__device__ void diag_tile(int s, int list_pos0, const double *__restrict__ T, int64_t ldt,
                          const Plan &P, const double *__restrict__ tau,
                          const double *__restrict__ blk_tau, double *__restrict__ Y, int64_t ldy,
                          int32_t *__restrict__ seg_e, double *__restrict__ seg_nu,
                          int32_t *__restrict__ seg_dx, int32_t *__restrict__ seg_dy,
                          double *smem, const Pencil &pen = Pencil(), bool decide = true) {
    constexpr int G = Lanes<C, GR>::G;
    constexpr int kThreads = 32 * W;
    constexpr int kUnits = Lanes<C, GR>::U * W;
    constexpr int ys = kUnits + 1;
    constexpr int FW = C ? 8 : 4;                      // factor doubles per block
    const int t0 = P.tile_start[s];
    const int ts = P.tile_start[s + 1] - t0;
    const int kb0 = P.tile_blk[s], kb1 = P.tile_blk[s + 1];
    const int nbt = kb1 - kb0;
    const int32_t *ord = C ? P.ord_cplx : P.ord_real;
    const int list_end = C ? P.ncplx : P.nreal;
    const int64_t m = P.m;
    const int tid = threadIdx.x;

    // shared layout
    double *Ts = smem;                                 // packed tile, pk_size(ts)
    double *btau = Ts + pk_size(ts);                   // [kMaxTile]
    double *umu = btau + kMaxTile;                     // [kUnits]
    double *yr = umu + kUnits;                         // [ts][ys]
    double *yi = yr + ts * ys;                         // [ts][ys], complex units only
    double *fac = yi + (C ? ts * ys : 0);              // [kUnits][ts][FW]
    int *bq = (int *)(fac + (size_t)kUnits * ts * FW); // [kMaxTile]
    int *bsz = bq + kMaxTile;                          // [kMaxTile]
    int *btf = bsz + kMaxTile;                         // [kMaxTile] exponent field of btau
    int *ford = btf + kMaxTile;                        // [kMaxTile] 1x1 blocks, then 2x2
    int *ucol = ford + kMaxTile;                       // [kUnits] column, -1 = none
    int *uown = ucol + kUnits;                         // [kUnits]
    int *ue = uown + kUnits;                           // [kUnits]
    int *facp = ue + kUnits;                           // [kUnits][ts] pivot positions
    int *uidx = facp + kUnits * ts;                    // [kUnits] unit index
    // pencils: T's tile, its in-tile block norms, per-unit block bounds
    double *Bt = (double *)(((uintptr_t)(uidx + kUnits) + 15) & ~(uintptr_t)15);   // packed
    double *btauB = Bt + (GEN ? pk_size(ts) : 0);      // [kMaxTile]
    double *utau = btauB + (GEN ? kMaxTile : 0);       // [kUnits][ts]

    // diagonal tile (upper part and first subdiagonal only), asynchronously
    for (int idx = tid; idx < ts * ts; idx += kThreads) {
        const int i = idx % ts, j = idx / ts;
        if (i <= j + 1) cp_async8(&Ts[pk_col(j) + i], T + (t0 + i) + (int64_t)(t0 + j) * ldt);
    }
    if constexpr (GEN)
        for (int idx = tid; idx < ts * ts; idx += kThreads) {
            const int i = idx % ts, j = idx / ts;
            if (i <= j) cp_async8(&Bt[pk_col(j) + i], pen.T + (t0 + i) + (int64_t)(t0 + j) * pen.ldt);
        }
    asm volatile("cp.async.commit_group;");
    for (int k = tid; k < nbt; k += kThreads) {
        bq[k] = P.blk_start[kb0 + k] - t0;
        bsz[k] = P.blk_size[kb0 + k];
    }
    if (tid < kUnits) {
        const int pos = list_pos0 + tid;
        int c = -1, own = 0, ui = 0;
        if (pos < list_end) {
            ui = ord[pos];
            c = P.unit_col[ui];
            own = P.unit_tile[ui] == s;
        }
        ucol[tid] = c;
        uown[tid] = own;
        uidx[tid] = ui;
    }
    __syncthreads();   // block list and unit map are read by every warp below
    if (tid == 0) {    // factor order: all 1x1 blocks, then all 2x2 blocks
        int f = 0;
        for (int k = 0; k < nbt; k++) if (bsz[k] == 1) ford[f++] = k;
        for (int k = 0; k < nbt; k++) if (bsz[k] == 2) ford[f++] = k;
    }
    // the tile, then the block factors below (they need only T and the
    // shifts: with a programmatic launch this part overlaps the previous
    // kernel of the stream)
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    // ---- one unit per G lanes --------------------------------------------
    const int slot = tid / G, g = tid % G;
    const int pos = list_pos0 + slot;
    const bool valid = pos < list_end;
    const int u = valid ? ord[pos] : 0;
    const int col = valid ? P.unit_col[u] : 0;
    const int kown = valid ? P.unit_blk[u] : -1;
    const bool own = valid && P.unit_tile[u] == s;
    const double lr = valid ? P.unit_lam[2 * u] : 0.0;
    const double li = (C && valid) ? P.unit_lam[2 * u + 1] : 0.0;
    const double be = (GEN && valid) ? P.unit_beta[u] : 1.0;
    const double smin = GEN ? (valid ? P.unit_smin[u] : 1.0)
                            : fmax(kUlp * (fabs(lr) + fabs(li)), kSafeMin * ((double)P.n / kUlp));
    double *myutau = utau + (size_t)slot * ts;
    double *myr = yr + slot;
    double *myi = yi + slot;
    double *myfac = fac + (size_t)slot * ts * FW;
    int *myfacp = facp + slot * ts;

    // factors of every block this unit solves, spread over its lanes in
    // size order (lanes of a warp take the same branch)
    if (valid) {
        for (int f = g; f < nbt; f += G) {
            const int kk = ford[f];
            if (own && kb0 + kk >= kown) continue;
            Fac F;
            if constexpr (GEN) {
                F = factor_pencil<C, true>(bsz[kk], Ts, Bt, ts, bq[kk], lr, li, be, smin);
            } else {
                F = factor<C, true>(bsz[kk], Ts, ts, bq[kk], lr, li, smin);
            }
            double *fp = myfac + kk * FW;
            if (C) {
                fp[0] = F.ia.re; fp[1] = F.ia.im; fp[2] = F.l.re; fp[3] = F.l.im;
                fp[4] = F.g.re;  fp[5] = F.g.im;  fp[6] = F.iu.re; fp[7] = F.iu.im;
            } else {
                fp[0] = F.ia.re; fp[1] = F.l.re; fp[2] = F.g.re; fp[3] = F.iu.re;
            }
            myfacp[kk] = F.pr | (F.pc << 1);
        }
    }

    // everything below reads what earlier kernels of the stream wrote (the
    // block norms, the segments and their exponents)
    grid_dependency_wait();
    for (int k = tid; k < nbt; k += kThreads) {
        btau[k] = blk_tau[kb0 + k];
        btf[k] = efield(blk_tau[kb0 + k]);
        if constexpr (GEN) btauB[k] = pen.blk_tau[kb0 + k];
    }
    // the segments, column by column (coalesced); own units start at zero
    for (int idx = tid; idx < kUnits * ts; idx += kThreads) {
        const int uu = idx / ts, i = idx % ts;
        const int c = ucol[uu];
        if (c >= 0 && (RHS || !uown[uu]) &&
            evec_in(P, t0 + i < P.n && c + (C ? 1 : 0) < P.m, 101)) {
            cp_async8(&yr[i * ys + uu], &Y[(t0 + i) + (int64_t)c * ldy]);
            if (C) cp_async8(&yi[i * ys + uu], &Y[(t0 + i) + (int64_t)(c + 1) * ldy]);
        } else {
            yr[i * ys + uu] = 0.0;
            if (C) yi[i * ys + uu] = 0.0;
        }
    }
    asm volatile("cp.async.commit_group;");
    if constexpr (GEN) {   // bound of the in-tile update from each block, this unit
        __syncthreads();
        if (valid)
            for (int f = g; f < nbt; f += G) {
                const int kk = ford[f];
                if (own && kb0 + kk >= kown) continue;
                myutau[kk] = fabs(be) * btau[kk] + (fabs(lr) + fabs(li)) * btauB[kk];
            }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    int e = 0;
    long long nbits = 0;
    if (valid && (RHS || !own)) {
        e = seg_e[(int64_t)s * m + col];
        for (int i = g; i < ts; i += G) {
            nbits = max(nbits, abs_bits(myr[i * ys]));
            if (C) nbits = max(nbits, abs_bits(myi[i * ys]));
        }
    }
    int Enu = efield(__longlong_as_double(group_max_bits<G>(nbits))) - 1022;   // nu < 2^Enu
    __syncwarp();

    auto scale_rows = [&](int k) {
        for (int i = g; i < ts; i += G) {
            myr[i * ys] = scale2(myr[i * ys], k);
            if (C) myi[i * ys] = scale2(myi[i * ys], k);
        }
    };

    // The update of the rows above a solved block is applied at the start of
    // the next block step (pending: block row pq, size pbs, solution pz0 /
    // pz1; pq <= 0 = none).  Each lane walks its own rows from the highest
    // down, so the next block's rows are updated first; their owner lanes
    // then hand them to the unit's other lanes by shuffle.  No lane reads
    // another lane's rows in shared memory, so the chain has no warp
    // barrier and no shared-memory round trip between the solves.
    int pq = 0, pbs = 1;
    Cx pz0 = {0.0, 0.0}, pz1 = {0.0, 0.0};
    for (int k = kb1 - 1; k >= kb0; k--) {
        const int kk = k - kb0;
        const int q = bq[kk];
        const int bs = bsz[kk];
        const double tauk = GEN ? myutau[kk] : btau[kk];
        const int ftq = GEN ? efield(tauk) : btf[kk];
        const bool act = valid && (!own || k <= kown);
        const bool solving = act && !(own && k == kown);
        if (pq > 0) {   // rows [0, pq) -= (block pq) pz; pq = q + bs
            const double *c0 = Ts + pk_col(pq);             // column pq, rows [0, pq)
            if constexpr (GEN) {
                const double *d0 = Bt + pk_col(pq);
                const Cx zb0 = {be * pz0.re, be * pz0.im}, zb1 = {be * pz1.re, be * pz1.im};
                const Cx wz0 = cmul<C>(Cx{lr, li}, pz0), wz1 = cmul<C>(Cx{lr, li}, pz1);
                if (pbs == 1)
                    update_rows_pencil<C, 1, G>(myr, myi, c0, c0, d0, d0, pq, g, zb0, zb1, wz0,
                                                wz1, ys);
                else
                    update_rows_pencil<C, 2, G>(myr, myi, c0, Ts + pk_col(pq + 1), d0,
                                                Bt + pk_col(pq + 1), pq, g, zb0, zb1, wz0, wz1,
                                                ys);
            } else {
                if (pbs == 1) update_rows<C, 1, G>(myr, myi, c0, c0, pq, g, pz0, pz1, ys);
                else update_rows<C, 2, G>(myr, myi, c0, Ts + pk_col(pq + 1), pq, g, pz0, pz1, ys);
            }
        }
        // the block's right-hand side from its owner lanes
        const int o0 = q % G, o1 = (q + 1) % G;
        double a0 = 0.0, b0 = 0.0, a1 = 0.0, b1 = 0.0;
        if (g == o0) {
            a0 = myr[q * ys];
            if (C) b0 = myi[q * ys];
        }
        if (bs == 2 && g == o1) {
            a1 = myr[(q + 1) * ys];
            if (C) b1 = myi[(q + 1) * ys];
        }
        Cx z0 = {0.0, 0.0}, z1 = {0.0, 0.0};
        const Cx r0 = {__shfl_sync(0xffffffffu, a0, o0, G),
                       C ? __shfl_sync(0xffffffffu, b0, o0, G) : 0.0};
        Cx r1 = {0.0, 0.0};
        if (bs == 2)
            r1 = {__shfl_sync(0xffffffffu, a1, o1, G), C ? __shfl_sync(0xffffffffu, b1, o1, G) : 0.0};
        Fac F;
        {
            const double *fp = myfac + kk * FW;
            if (C) {
                F.ia = {fp[0], fp[1]};
                F.l = {fp[2], fp[3]};
                F.g = {fp[4], fp[5]};
                F.iu = {fp[6], fp[7]};
            } else {
                F.ia = {fp[0], 0.0};
                F.l = {fp[1], 0.0};
                F.g = {fp[2], 0.0};
                F.iu = {fp[3], 0.0};
            }
            const int pp = myfacp[kk];
            F.pr = pp & 1;
            F.pc = pp >> 1;
        }
        if (act) {
            int sc = 0;
            if (!solving) {
                if (RHS) {   // the own block stays fixed: its correction is zero
                    z0 = {0.0, 0.0};
                    z1 = {0.0, 0.0};
                } else {
                    const double *o = P.unit_own + 4 * u;
                    z0 = {o[0], C ? o[2] : 0.0};
                    z1 = {o[1], C ? o[3] : 0.0};
                }
            } else {
                sc = solve<C>(F, bs, r0, r1, z0, z1, (g & 1) != 0, unit_mask<G>());
            }
            if (sc != 0) {
                scale_rows(sc);
                Enu += sc;
                e += sc;
            }
            if (g == o0) { myr[q * ys] = z0.re; if (C) myi[q * ys] = z0.im; }
            if (bs == 2 && g == o1) {
                myr[(q + 1) * ys] = z1.re;
                if (C) myi[(q + 1) * ys] = z1.im;
            }
        }
        // protection of the update of rows [0, q): fast test on exponents,
        // exact FP64 test only when it cannot decide (the rows already hold
        // every earlier block's update)
        int fmu = max(max(efield(z0.re), efield(z0.im)), max(efield(z1.re), efield(z1.im)));
        const bool trig = act && q > 0 && (Enu > 1019 || fmu + ftq > 3063);
        if (__any_sync(0xffffffffu, trig)) {
            long long b = 0;
            if (trig)
                for (int i = g; i < q; i += G) {
                    b = max(b, abs_bits(myr[i * ys]));
                    if (C) b = max(b, abs_bits(myi[i * ys]));
                }
            b = group_max_bits<G>(b);
            if (trig) {
                double nu = __longlong_as_double(b);
                const double mu = __longlong_as_double(max(cbits(z0), cbits(z1)));
                const int g2 = protect_update(nu, tauk, mu);
                if (g2 != 0) {
                    scale_rows(g2);
                    z0 = cscale(z0, g2);
                    z1 = cscale(z1, g2);
                    nu = scale2(nu, g2);
                    e += g2;
                    fmu = max(max(efield(z0.re), efield(z0.im)), max(efield(z1.re), efield(z1.im)));
                }
                Enu = efield(nu) - 1022;
            }
        }
        // the update with this block's z runs at the start of the next step
        if (act && q > 0) {
            pq = q;
            pbs = bs;
            pz0 = z0;
            pz1 = z1;
            Enu = max(Enu, fmu + ftq - 2044) + 1;
        } else {
            pq = 0;
        }
    }
    __syncwarp();
    // segment maxima per column, exponent
    {
        long long br = 0, bi = 0;
        for (int i = g; i < ts; i += G) {
            br = max(br, abs_bits(myr[i * ys]));
            if (C) bi = max(bi, abs_bits(myi[i * ys]));
        }
        br = group_max_bits<G>(br);
        bi = group_max_bits<G>(bi);
        if (g == 0) {
            ue[slot] = e;
            umu[slot] = __longlong_as_double(max(br, bi));
            if (valid) {
                seg_e[(int64_t)s * m + col] = e;
                seg_nu[(int64_t)s * m + col] = __longlong_as_double(br);
                if (C) {
                    seg_e[(int64_t)s * m + col + 1] = e;
                    seg_nu[(int64_t)s * m + col + 1] = __longlong_as_double(bi);
                }
            }
        }
    }
    __syncthreads();

    // ---- write-back and the decisions for the tiles above ------------------
    for (int idx = tid; idx < kUnits * ts; idx += kThreads) {
        const int uu = idx / ts, i = idx % ts;
        const int c = ucol[uu];
        if (c >= 0 && evec_in(P, t0 + i < P.n && c + (C ? 1 : 0) < P.m, 102)) {
            Y[(t0 + i) + (int64_t)c * ldy] = yr[i * ys + uu];
            if (C) Y[(t0 + i) + (int64_t)(c + 1) * ldy] = yi[i * ys + uu];
        }
    }
    // consolidation + protection decisions (Sec. 3.3): thread -> (unit,
    // tile row), consecutive threads on consecutive columns; four items per
    // thread per round so their loads are in flight together
    // (decide == false: a separate launch takes them, k_decide)
    constexpr int kBatch = 4;
    const int items = decide ? kUnits * s : 0;
    for (int base = tid; base < items; base += kBatch * kThreads) {
        int er[kBatch];
        double nur[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; j++) {
            const int idx = base + j * kThreads;
            er[j] = 0;
            nur[j] = 0.0;
            if (idx < items) {
                const int uu = idx % kUnits, r = idx / kUnits;
                const int c = ucol[uu];
                if (c >= 0 && (RHS || !uown[uu]) &&
                    evec_in(P, r < P.ntiles && c + (C ? 1 : 0) < m, 103)) {
                    const int64_t at = (int64_t)r * m + c;
                    er[j] = seg_e[at];
                    nur[j] = seg_nu[at];
                    if (C) nur[j] = fmax(nur[j], seg_nu[at + 1]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kBatch; j++) {
            const int idx = base + j * kThreads;
            if (idx >= items) continue;
            const int uu = idx % kUnits, r = idx / kUnits;
            const int c = ucol[uu];
            if (c < 0 || !evec_in(P, r < P.ntiles && c + (C ? 1 : 0) < m, 104)) continue;
            const int64_t at = (int64_t)r * m + c;
            const int es = ue[uu];
            const bool ownu = !RHS && uown[uu];   // fresh segments above the own block
            const int e_r = ownu ? es : er[j];
            const int a = min(e_r, es);
            double trs = tau[(int64_t)r * P.ntiles + s];
            if constexpr (GEN) {   // |beta| |S_rs| + |alpha|_1 |T_rs| for this unit
                const int ui = uidx[uu];
                trs = fabs(P.unit_beta[ui]) * trs +
                      (fabs(P.unit_lam[2 * ui]) + fabs(P.unit_lam[2 * ui + 1])) *
                          pen.tau[(int64_t)r * P.ntiles + s];
            }
            const int g2 = protect_update_scaled(ownu ? 0.0 : nur[j], a - e_r, trs, umu[uu], a - es);
            const int ne = a + g2;
            seg_e[at] = ne;
            seg_dx[at] = ne - es;
            seg_dy[at] = ownu ? kFresh : ne - e_r;
            seg_nu[at] = 0.0;   // the update of this step writes the new maximum
            if (C) {
                seg_e[at + 1] = ne;
                seg_dx[at + 1] = ne - es;
                seg_dy[at + 1] = ownu ? kFresh : ne - e_r;
                seg_nu[at + 1] = 0.0;
            }
        }
    }
}

}  // namespace

// dynamic shared memory of diag_tile<W, C, GEN, *, GR> for a tile of t rows
template <int W, bool C, bool GEN = false, int GR = 8>
inline size_t diag_smem_bytes(int t) {
    constexpr int kUnits = Lanes<C, GR>::U * W;
    constexpr int FW = C ? 8 : 4;
    return sizeof(double) * ((size_t)pk_size(t) + kMaxTile + kUnits +
                             (C ? 2 : 1) * (size_t)t * (kUnits + 1) + (size_t)kUnits * t * FW) +
           sizeof(int) * (4 * (size_t)kMaxTile + 4 * kUnits + (size_t)kUnits * t) + 16 +
           (GEN ? sizeof(double) * ((size_t)pk_size(t) + kMaxTile + (size_t)kUnits * t) : 0);
}

template <int W, bool GEN = false, int GR = 8>
inline size_t diag_smem(int t) {
    return std::max(diag_smem_bytes<W, false, GEN, GR>(t), diag_smem_bytes<W, true, GEN, GR>(t));
}

}  // namespace evec
