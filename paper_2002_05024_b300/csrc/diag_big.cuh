// diag_big.cuh -- the robust diagonal-tile solve for tiles of more than 64
// rows (up to kMaxTileBig), as a device function for the per-step kernel
// (k_diag_solve.cu).
//
// A tile of this size does not fit in shared memory, but every unit's
// segment of it does (one scale exponent per tile segment, as for every
// tile: the augmented tile of Sec. 3.3).  The tile is walked in sub-blocks
// of at most 64 rows from the bottom (boundaries moved up one row where
// they would split a 2x2 block).  For sub-block j (tile rows [a, b)):
//   1. its diagonal part T[a:b, a:b] is staged in shared memory and the
//      factors of its shifted 1x1 / 2x2 block systems are computed (the
//      same device code as the 64-row tiles);
//   2. the chain of block solves runs over the sub-block exactly as in a
//      64-row tile, its updates restricted to the sub-block's rows;
//   3. the rows above, [0, a), get the sub-block's contribution in one
//      pass, rows -= T[0:a, a:b] z, with T staged 64 rows at a time.  It is
//      protected like any update: nu = max |rows [0, a)|, tau = sum of the
//      in-tile block column norms of the sub-block's blocks (an upper bound
//      of ||T[0:a, a:b]||_inf: each block norm covers all rows above its
//      block), mu = max |z| over the sub-block; a scaling 2^q of the whole
//      segment keeps nu + tau mu <= Omega, so no partial sum overflows in
//      any order.
// The maxima, write-back and the decisions for the tiles above are those
// of the 64-row tiles.
// GEN (a pencil beta S - alpha T, T upper triangular): S takes T's place
// above, T's sub-block and panels are staged beside S's, the chain runs the
// pencil updates, the pass over the rows above subtracts
// S[0:a, a:b] (beta z) - T[0:a, a:b] (alpha z), and every bound is
// |beta| |S ..| + |alpha|_1 |T ..|.
#pragma once

#include "diag_tile.cuh"

namespace evec {

namespace {

constexpr int kSub = 64;                                 // rows of a sub-block, at most
constexpr int kMaxSubs = kMaxTileBig / (kSub - 1) + 2;   // sub-blocks of a tile, at most

template <int W, bool C, bool GEN, bool RHS, int GR = 8>
__device__ void diag_tile_big(int s, int list_pos0, const double *__restrict__ T, int64_t ldt,
                              const Plan &P, const double *__restrict__ tau,
                              const double *__restrict__ blk_tau, double *__restrict__ Y,
                              int64_t ldy, int32_t *__restrict__ seg_e,
                              double *__restrict__ seg_nu, int32_t *__restrict__ seg_dx,
                              int32_t *__restrict__ seg_dy, double *smem, bool decide,
                              const Pencil &pen = Pencil()) {
    constexpr int G = Lanes<C, GR>::G;
    constexpr int kThreads = 32 * W;
    constexpr int kUnits = Lanes<C, GR>::U * W;
    constexpr int ys = kUnits + 1;
    constexpr int FW = C ? 8 : 4;                      // factor doubles per block
    constexpr int R = (kSub + G - 1) / G;              // rows per lane of a 64-row chunk
    const int t0 = P.tile_start[s];
    const int ts = P.tile_start[s + 1] - t0;
    const int kb0 = P.tile_blk[s], kb1 = P.tile_blk[s + 1];
    const int nbt = kb1 - kb0;
    const int32_t *ord = C ? P.ord_cplx : P.ord_real;
    const int list_end = C ? P.ncplx : P.nreal;
    const int64_t m = P.m;
    const int tid = threadIdx.x;

    // shared layout
    double *Tsub = smem;                               // kSub x kSub, ld kSub (also T panels)
    double *btau = Tsub + kSub * kSub;                 // [ts] block column norms
    double *stau = btau + ts;                          // [kMaxSubs] sub-block panel bounds
    double *umu = stau + kMaxSubs;                     // [kUnits]
    double *yr = umu + kUnits;                         // [ts][ys]
    double *yi = yr + ts * ys;                         // [ts][ys], complex units only
    double *fac = yi + (C ? ts * ys : 0);              // [kUnits][kSub][FW]
    int *bq = (int *)(fac + (size_t)kUnits * kSub * FW);   // [ts] block rows (tile-local)
    int *bsz = bq + ts;                                // [ts]
    int *btf = bsz + ts;                               // [ts] exponent field of btau
    int *ford = btf + ts;                              // [kSub] factor order of a sub-block
    int *ucol = ford + kSub;                           // [kUnits] column, -1 = none
    int *uown = ucol + kUnits;                         // [kUnits]
    int *ue = uown + kUnits;                           // [kUnits]
    int *facp = ue + kUnits;                           // [kUnits][kSub] pivot positions
    int *srow = facp + kUnits * kSub;                  // [kMaxSubs + 1] sub-block rows
    int *sblk = srow + kMaxSubs + 1;                   // [kMaxSubs + 1] sub-block first blocks
    int *snsub = sblk + kMaxSubs + 1;                  // [1]
    // pencils: T's sub-block (and T panels), its block norms, the bounds of
    // the sub-blocks' T panels, per-unit block bounds
    double *Bsub = (double *)(((uintptr_t)(snsub + 1) + 15) & ~(uintptr_t)15);   // kSub x kSub
    double *btauB = Bsub + (GEN ? kSub * kSub : 0);    // [ts]
    double *stauB = btauB + (GEN ? ts : 0);            // [kMaxSubs]
    double *utau = stauB + (GEN ? kMaxSubs : 0);       // [kUnits][kSub]

    // the block norms and segments come from earlier kernels of the stream
    grid_dependency_wait();
    for (int k = tid; k < nbt; k += kThreads) {
        bq[k] = P.blk_start[kb0 + k] - t0;
        bsz[k] = P.blk_size[kb0 + k];
        btau[k] = blk_tau[kb0 + k];
        btf[k] = efield(blk_tau[kb0 + k]);
        if constexpr (GEN) btauB[k] = pen.blk_tau[kb0 + k];
    }
    if (tid < kUnits) {
        const int pos = list_pos0 + tid;
        int c = -1, own = 0;
        if (pos < list_end) {
            const int ui = ord[pos];
            c = P.unit_col[ui];
            own = P.unit_tile[ui] == s;
        }
        ucol[tid] = c;
        uown[tid] = own;
    }
    __syncthreads();   // block list and unit map are read by every warp below
    if (tid == 0) {
        // sub-blocks of at most kSub rows from the top; a boundary that
        // would split a 2x2 block moves up one row
        int ns = 0, a = 0, k = 0;
        while (a < ts) {
            int b = a + kSub;
            if (b >= ts) {
                b = ts;
            } else {
                int kb = k;   // the block holding row b
                while (kb + 1 < nbt && bq[kb + 1] <= b) kb++;
                if (bq[kb] < b && bq[kb] + bsz[kb] > b) b = bq[kb];
            }
            srow[ns] = a;
            sblk[ns] = k;
            double tsum = 0.0, tsumB = 0.0;
            while (k < nbt && bq[k] < b) {
                tsum += btau[k];
                if constexpr (GEN) tsumB += btauB[k];
                k++;
            }
            stau[ns] = tsum;
            if constexpr (GEN) stauB[ns] = tsumB;
            ns++;
            a = b;
        }
        srow[ns] = ts;
        sblk[ns] = nbt;
        *snsub = ns;
    }
    // the segments, column by column (coalesced); own units start at zero
    for (int idx = tid; idx < kUnits * ts; idx += kThreads) {
        const int uu = idx / ts, i = idx % ts;
        const int c = ucol[uu];
        if (c >= 0 && (RHS || !uown[uu]) &&
            evec_in(P, t0 + i < P.n && c + (C ? 1 : 0) < P.m, 111)) {
            cp_async8(&yr[i * ys + uu], &Y[(t0 + i) + (int64_t)c * ldy]);
            if (C) cp_async8(&yi[i * ys + uu], &Y[(t0 + i) + (int64_t)(c + 1) * ldy]);
        } else {
            yr[i * ys + uu] = 0.0;
            if (C) yi[i * ys + uu] = 0.0;
        }
    }
    asm volatile("cp.async.commit_group;");
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
    double *myutau = utau + (size_t)slot * kSub;
    double *myr = yr + slot;
    double *myi = yi + slot;
    double *myfac = fac + (size_t)slot * kSub * FW;
    int *myfacp = facp + slot * kSub;
    const int nsub = *snsub;

    int e = 0;
    if (valid && (RHS || !own)) e = seg_e[(int64_t)s * m + col];

    auto scale_rows = [&](int k) {
        for (int i = g; i < ts; i += G) {
            myr[i * ys] = scale2(myr[i * ys], k);
            if (C) myi[i * ys] = scale2(myi[i * ys], k);
        }
    };
    // max |y| over the unit's rows [r0, r1), as a bit pattern
    auto rows_max = [&](int r0, int r1) -> long long {
        long long b = 0;
        for (int i = r0 + g; i < r1; i += G) {
            b = max(b, abs_bits(myr[i * ys]));
            if (C) b = max(b, abs_bits(myi[i * ys]));
        }
        return group_max_bits<G>(b);
    };

    for (int j = nsub - 1; j >= 0; j--) {
        const int a = srow[j], b = srow[j + 1];
        const int sb0 = sblk[j], sb1 = sblk[j + 1];   // the sub-block's blocks
        const int nsb = sb1 - sb0;
        const int sts = b - a;                       // rows of the sub-block
        // ---- 1. the sub-block's diagonal part and its block factors -----
        __syncthreads();   // every reader of Tsub / ford (previous sub-block) is done
        for (int idx = tid; idx < kSub * kSub; idx += kThreads) {
            const int i = idx % kSub, jj = idx / kSub;
            if (i < sts && jj < sts && i <= jj + 1)
                cp_async8(&Tsub[idx], T + (t0 + a + i) + (int64_t)(t0 + a + jj) * ldt);
            else Tsub[idx] = 0.0;
            if constexpr (GEN) {
                if (i < sts && jj < sts && i <= jj)
                    cp_async8(&Bsub[idx],
                              pen.T + (t0 + a + i) + (int64_t)(t0 + a + jj) * pen.ldt);
                else Bsub[idx] = 0.0;
            }
        }
        asm volatile("cp.async.commit_group;");
        if (tid == 0) {   // factor order: the 1x1 blocks, then the 2x2 blocks
            int f = 0;
            for (int k = 0; k < nsb; k++) if (bsz[sb0 + k] == 1) ford[f++] = k;
            for (int k = 0; k < nsb; k++) if (bsz[sb0 + k] == 2) ford[f++] = k;
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (valid) {
            for (int f = g; f < nsb; f += G) {
                const int kl = ford[f];
                if (own && kb0 + sb0 + kl >= kown) continue;
                Fac F;
                if constexpr (GEN) {
                    F = factor_pencil<C>(bsz[sb0 + kl], Tsub, Bsub, kSub, bq[sb0 + kl] - a, lr, li,
                                         be, smin);
                    myutau[kl] = fabs(be) * btau[sb0 + kl] + (fabs(lr) + fabs(li)) * btauB[sb0 + kl];
                } else {
                    F = factor<C>(bsz[sb0 + kl], Tsub, kSub, bq[sb0 + kl] - a, lr, li, smin);
                }
                double *fp = myfac + kl * FW;
                if (C) {
                    fp[0] = F.ia.re; fp[1] = F.ia.im; fp[2] = F.l.re; fp[3] = F.l.im;
                    fp[4] = F.g.re;  fp[5] = F.g.im;  fp[6] = F.iu.re; fp[7] = F.iu.im;
                } else {
                    fp[0] = F.ia.re; fp[1] = F.l.re; fp[2] = F.g.re; fp[3] = F.iu.re;
                }
                myfacp[kl] = F.pr | (F.pc << 1);
            }
        }
        __syncwarp();   // the unit's lanes read each other's factors below

        // ---- 2. the chain of block solves over the sub-block ------------
        // local rows: row i of the sub-block is tile row a + i
        double *lyr = myr + a * ys;
        double *lyi = myi + a * ys;
        int Enu = efield(__longlong_as_double(rows_max(a, b))) - 1022;   // nu < 2^Enu
        auto scale_all = [&](int k) { scale_rows(k); };
        int pq = 0, pbs = 1;
        Cx pz0 = {0.0, 0.0}, pz1 = {0.0, 0.0};
        for (int kl = nsb - 1; kl >= 0; kl--) {
            const int kt = sb0 + kl;                 // block index within the tile
            const int k = kb0 + kt;                  // global block index
            const int q = bq[kt] - a;                // local row of the block
            const int bs = bsz[kt];
            const double tauk = GEN ? myutau[kl] : btau[kt];
            const int ftq = GEN ? efield(tauk) : btf[kt];
            const bool act = valid && (!own || k <= kown);
            const bool solving = act && !(own && k == kown);
            if (pq > 0) {   // local rows [0, pq) -= (block pq) pz
                const double *c0 = Tsub + pq * kSub;
                if constexpr (GEN) {
                    const double *d0 = Bsub + pq * kSub;
                    const Cx zb0 = {be * pz0.re, be * pz0.im}, zb1 = {be * pz1.re, be * pz1.im};
                    const Cx wz0 = cmul<C>(Cx{lr, li}, pz0), wz1 = cmul<C>(Cx{lr, li}, pz1);
                    if (pbs == 1)
                        update_rows_pencil<C, 1, G>(lyr, lyi, c0, c0, d0, d0, pq, g, zb0, zb1, wz0,
                                                    wz1, ys);
                    else
                        update_rows_pencil<C, 2, G>(lyr, lyi, c0, c0 + kSub, d0, d0 + kSub, pq, g,
                                                    zb0, zb1, wz0, wz1, ys);
                } else {
                    if (pbs == 1) update_rows<C, 1, G>(lyr, lyi, c0, c0, pq, g, pz0, pz1, ys);
                    else update_rows<C, 2, G>(lyr, lyi, c0, c0 + kSub, pq, g, pz0, pz1, ys);
                }
            }
            const int o0 = q % G, o1 = (q + 1) % G;
            double a0 = 0.0, b0 = 0.0, a1 = 0.0, b1 = 0.0;
            if (g == o0) {
                a0 = lyr[q * ys];
                if (C) b0 = lyi[q * ys];
            }
            if (bs == 2 && g == o1) {
                a1 = lyr[(q + 1) * ys];
                if (C) b1 = lyi[(q + 1) * ys];
            }
            Cx z0 = {0.0, 0.0}, z1 = {0.0, 0.0};
            const Cx r0 = {__shfl_sync(0xffffffffu, a0, o0, G),
                           C ? __shfl_sync(0xffffffffu, b0, o0, G) : 0.0};
            Cx r1 = {0.0, 0.0};
            if (bs == 2)
                r1 = {__shfl_sync(0xffffffffu, a1, o1, G),
                      C ? __shfl_sync(0xffffffffu, b1, o1, G) : 0.0};
            Fac F;
            {
                const double *fp = myfac + kl * FW;
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
                const int pp = myfacp[kl];
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
                    scale_all(sc);
                    Enu += sc;
                    e += sc;
                }
                if (g == o0) { lyr[q * ys] = z0.re; if (C) lyi[q * ys] = z0.im; }
                if (bs == 2 && g == o1) {
                    lyr[(q + 1) * ys] = z1.re;
                    if (C) lyi[(q + 1) * ys] = z1.im;
                }
            }
            // protection of the update of the sub-block's rows [0, q)
            int fmu = max(max(efield(z0.re), efield(z0.im)), max(efield(z1.re), efield(z1.im)));
            const bool trig = act && q > 0 && (Enu > 1019 || fmu + ftq > 3063);
            if (__any_sync(0xffffffffu, trig)) {
                long long bb = 0;
                if (trig)
                    for (int i = g; i < q; i += G) {
                        bb = max(bb, abs_bits(lyr[i * ys]));
                        if (C) bb = max(bb, abs_bits(lyi[i * ys]));
                    }
                bb = group_max_bits<G>(bb);
                if (trig) {
                    double nu = __longlong_as_double(bb);
                    const double mu = __longlong_as_double(max(cbits(z0), cbits(z1)));
                    const int g2 = protect_update(nu, tauk, mu);
                    if (g2 != 0) {
                        scale_all(g2);
                        z0 = cscale(z0, g2);
                        z1 = cscale(z1, g2);
                        nu = scale2(nu, g2);
                        e += g2;
                        fmu = max(max(efield(z0.re), efield(z0.im)),
                                  max(efield(z1.re), efield(z1.im)));
                    }
                    Enu = efield(nu) - 1022;
                }
            }
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

        // ---- 3. the rows above the sub-block -----------------------------
        if (a == 0) continue;
        {   // protection: nu = max |rows [0, a)|, tau = stau[j], mu = max |z|
            const double nu = __longlong_as_double(rows_max(0, a));
            const double mu = __longlong_as_double(rows_max(a, b));
            const double tb = GEN ? fabs(be) * stau[j] + (fabs(lr) + fabs(li)) * stauB[j]
                                  : stau[j];
            const int g2 = valid ? protect_update(nu, tb, mu) : 0;
            if (g2 != 0) {
                scale_rows(g2);
                e += g2;
            }
        }
        __syncwarp();
        for (int c0 = 0; c0 < a; c0 += kSub) {
            const int rows = min(kSub, a - c0);
            __syncthreads();   // the chain's (or the previous chunk's) reads of Tsub are done
            for (int idx = tid; idx < kSub * sts; idx += kThreads) {
                const int i = idx % kSub, c = idx / kSub;   // Tsub[c][i] = T[c0 + i, a + c]
                if (i < rows) {
                    cp_async8(&Tsub[c * kSub + i], T + (t0 + c0 + i) + (int64_t)(t0 + a + c) * ldt);
                    if constexpr (GEN)
                        cp_async8(&Bsub[c * kSub + i],
                                  pen.T + (t0 + c0 + i) + (int64_t)(t0 + a + c) * pen.ldt);
                }
            }
            asm volatile("cp.async.commit_group;");
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            double accr[R], acci[R];
#pragma unroll
            for (int t = 0; t < R; t++) {
                accr[t] = 0.0;
                acci[t] = 0.0;
            }
            for (int c = 0; c < sts; c++) {
                const double zr = myr[(a + c) * ys];
                const double zi = C ? myi[(a + c) * ys] : 0.0;
                const double *tc = Tsub + c * kSub;
                if constexpr (GEN) {
                    // rows -= S (beta z) - T (alpha z): accumulate
                    // S zb - T wz with zb = beta z, wz = alpha z
                    const Cx zb = {be * zr, be * zi};
                    const Cx wz = cmul<C>(Cx{lr, li}, Cx{zr, zi});
                    const double *dc = Bsub + c * kSub;
#pragma unroll
                    for (int t = 0; t < R; t++) {
                        const int i = g + G * t;
                        if (i < rows) {
                            const double sv = tc[i], tv = dc[i];
                            accr[t] = fma(-tv, wz.re, fma(sv, zb.re, accr[t]));
                            if (C) acci[t] = fma(-tv, wz.im, fma(sv, zb.im, acci[t]));
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < R; t++) {
                        const int i = g + G * t;
                        if (i < rows) {
                            const double tv = tc[i];
                            accr[t] = fma(tv, zr, accr[t]);
                            if (C) acci[t] = fma(tv, zi, acci[t]);
                        }
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < R; t++) {
                const int i = g + G * t;
                if (i < rows) {
                    myr[(c0 + i) * ys] -= accr[t];
                    if (C) myi[(c0 + i) * ys] -= acci[t];
                }
            }
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
        if (c >= 0 && evec_in(P, t0 + i < P.n && c + (C ? 1 : 0) < P.m, 112)) {
            Y[(t0 + i) + (int64_t)c * ldy] = yr[i * ys + uu];
            if (C) Y[(t0 + i) + (int64_t)(c + 1) * ldy] = yi[i * ys + uu];
        }
    }
    const int items = decide ? kUnits * s : 0;
    for (int idx = tid; idx < items; idx += kThreads) {
        const int uu = idx % kUnits, r = idx / kUnits;
        const int c = ucol[uu];
        if (c < 0 || !evec_in(P, r < P.ntiles && c + (C ? 1 : 0) < m, 113)) continue;
        const int64_t at = (int64_t)r * m + c;
        const int es = ue[uu];
        const bool ownu = !RHS && uown[uu];   // fresh segments above the own block
        const int e_r = ownu ? es : seg_e[at];
        double nur = 0.0;
        if (!ownu) {
            nur = seg_nu[at];
            if (C) nur = fmax(nur, seg_nu[at + 1]);
        }
        const int aa = min(e_r, es);
        double trs = tau[(int64_t)r * P.ntiles + s];
        if constexpr (GEN) {   // |beta| |S_rs| + |alpha|_1 |T_rs| for this unit
            const int ui = ord[list_pos0 + uu];
            trs = fabs(P.unit_beta[ui]) * trs +
                  (fabs(P.unit_lam[2 * ui]) + fabs(P.unit_lam[2 * ui + 1])) *
                      pen.tau[(int64_t)r * P.ntiles + s];
        }
        const int g2 = protect_update_scaled(nur, aa - e_r, trs, umu[uu], aa - es);
        const int ne = aa + g2;
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

}  // namespace

// dynamic shared memory of diag_tile_big<W, C, *, GR> for a tile of t rows
template <int W, bool C, bool GEN = false, int GR = 8>
inline size_t diag_big_smem_bytes(int t) {
    constexpr int kUnits = Lanes<C, GR>::U * W;
    constexpr int FW = C ? 8 : 4;
    return sizeof(double) * ((size_t)kSub * kSub + (size_t)t + kMaxSubs + kUnits +
                             (C ? 2 : 1) * (size_t)t * (kUnits + 1) +
                             (size_t)kUnits * kSub * FW) +
           sizeof(int) * (3 * (size_t)t + kSub + 3 * kUnits + (size_t)kUnits * kSub +
                          2 * (kMaxSubs + 1) + 1) + 16 +
           (GEN ? sizeof(double) * ((size_t)kSub * kSub + (size_t)t + kMaxSubs +
                                    (size_t)kUnits * kSub)
                : 0);
}

template <int W, bool GEN = false, int GR = 8>
inline size_t diag_big_smem(int t) {
    return std::max(diag_big_smem_bytes<W, false, GEN, GR>(t),
                    diag_big_smem_bytes<W, true, GEN, GR>(t));
}

}  // namespace evec
