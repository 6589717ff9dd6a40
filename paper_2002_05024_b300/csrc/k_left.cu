// k_left.cu -- left eigenvectors through the flipped Schur form.
//
// A left eigenvector u of T (u^H T = lambda u^H, Sec. 2's eigenvector
// problem for T^T) satisfies T^T conj(u) = lambda conj(u).  With J the
// reversal permutation, T' = J T^T J is again upper quasi-triangular with
// the same 1x1 / 2x2 blocks in reverse order (a standardized block
// [[a, b], [c, a]] maps to itself), so conj(u) = J y' for the right
// eigenvector y' of T' and the whole right-eigenvector path runs unchanged
// on T'.  These kernels move the data in and out of that form: T' itself,
// Q J for the back-transformation (Q u = (Q J) conj-free y'), and the final
// scatter that restores T's column order, reverses the rows (without Q)
// and negates the imaginary columns (u = conj(J y')).  All three are plain
// copies: HBM-bound, one read and one write per element.
//
// Pencils: the left eigenvectors of (S, T), u^H (beta S - alpha T) = 0, are
// the reversed conjugated right eigenvectors of (J S^T J, J T^T J), again an
// upper quasi-triangular S' over an upper triangular T' with the same
// blocks in reverse order (a diagonal 2x2 block of T stays diagonal), so
// the same three copies serve there, with T' flipped without a subdiagonal.
#include <algorithm>

#include "evec_internal.cuh"

namespace evec {

constexpr int kFlipTile = 32;

// T'(i, j) = T(n-1-j, n-1-i) for j >= i - sub (sub = 1: the part the
// solver reads, upper triangle and first subdiagonal, T's own referenced
// part mirrored; sub = 0: the upper triangle of a pencil's triangular
// factor), zero below.  One 32 x 32 tile of T' per CTA (32 x 8 threads) through
// shared memory, so that both the reads of T (along its columns) and the
// writes of T' are coalesced.  Entries of T strictly above its first
// superdiagonal are validated here (finite, <= 2^1000) and reported in T's
// own coordinates (r + c ldt) before the solve on T' sees them; the three
// central diagonals are validated by the planner.
__global__ void __launch_bounds__(256)
    k_flip_transpose(const double *__restrict__ T, int64_t ldt, int64_t n,
                     double *__restrict__ Tf, int64_t ldf, int sub, DevStatus *status) {
    __shared__ double tile[kFlipTile][kFlipTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i0 = (int64_t)blockIdx.y * kFlipTile;   // rows of T'
    const int64_t j0 = (int64_t)blockIdx.x * kFlipTile;   // columns of T'
    // whole tile strictly below the first subdiagonal of T': zeros
    const bool below = j0 + kFlipTile - 1 < i0 - sub;
    if (!below) {
        // load: lane tx reads T row r = n-1-(j0+31-tx) (consecutive r along
        // the lanes), column c = n-1-(i0+il)
        const int64_t jp = j0 + (kFlipTile - 1) - tx;
        for (int il = ty; il < kFlipTile; il += 8) {
            const int64_t ip = i0 + il;
            double v = 0.0;
            if (ip < n && jp < n && jp >= ip - sub) {
                const int64_t r = n - 1 - jp, c = n - 1 - ip;
                v = T[r + c * ldt];
                if (c >= r + 2) {
                    if (!isfinite(v)) report(status, 3 /* EVEC_ENONFINITE */, r + c * ldt);
                    else if (fabs(v) > kInputMax) report(status, 1 /* EVEC_EINVAL */, r + c * ldt);
                }
            }
            tile[il][(kFlipTile - 1) - tx] = v;
        }
    }
    __syncthreads();
    // store: lane tx writes T' row i0+tx of column j0+jl
    const int64_t ip = i0 + tx;
    if (ip >= n) return;
    for (int jl = ty; jl < kFlipTile; jl += 8) {
        const int64_t jp = j0 + jl;
        if (jp >= n) break;
        Tf[ip + jp * ldf] = below ? 0.0 : tile[tx][jl];
    }
}

// Qr(:, j) = Q(:, n-1-j): the back-transformation matrix of the flipped
// problem (Q J).
__global__ void __launch_bounds__(256)
    k_reverse_cols(const double *__restrict__ Q, int64_t ldq, int64_t n, int64_t j0,
                   double *__restrict__ Qr, int64_t ldr) {
    const int64_t j = j0 + blockIdx.y;
    const double *src = Q + (n - 1 - j) * ldq;
    double *dst = Qr + j * ldr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// X(:, d) = +-Xw(rows, c') for the source column c' = c0 + blockIdx.y,
// d = dst[c'] (or ~dst[c'] for a negated, imaginary column); rows reversed
// when `reverse` (no back-transformation), with the exponent and
// eigenvalue (and a pencil's beta) of the column carried along.
__global__ void __launch_bounds__(256)
    k_left_output(const double *__restrict__ Xw, int64_t ldw, int64_t n, int64_t c0,
                  const int32_t *__restrict__ dst, int reverse, const int32_t *__restrict__ ew,
                  const double *__restrict__ lrw, const double *__restrict__ liw,
                  double *__restrict__ X, int64_t ldx, int32_t *__restrict__ e,
                  double *__restrict__ lr, double *__restrict__ li,
                  const double *__restrict__ bw, double *__restrict__ bo) {
    const int64_t c = c0 + blockIdx.y;
    const int32_t code = dst[c];
    const bool neg = code < 0;
    const int64_t d = neg ? ~code : code;
    const double *src = Xw + c * ldw;
    double *out = X + d * ldx;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[reverse ? n - 1 - i : i];
        out[i] = neg ? -v : v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        e[d] = ew[c];
        if (lr) lr[d] = lrw[c];
        if (li) li[d] = liw[c];
        if (bo) bo[d] = bw[c];
    }
}

void launch_flip_transpose(const double *T, int64_t ldt, int64_t n, double *Tf, int64_t ldf,
                           DevStatus *status, cudaStream_t st, int sub) {
    if (n <= 0) return;
    const int64_t nt = (n + kFlipTile - 1) / kFlipTile;   // <= 65535 for n < 2^21
    k_flip_transpose<<<dim3((unsigned)nt, (unsigned)nt), dim3(kFlipTile, 8), 0, st>>>(
        T, ldt, n, Tf, ldf, sub, status);
}

void launch_reverse_cols(const double *Q, int64_t ldq, int64_t n, double *Qr, int64_t ldr,
                         cudaStream_t st) {
    if (n <= 0) return;
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 16);
    for (int64_t j0 = 0; j0 < n; j0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(n - j0, 65535);
        k_reverse_cols<<<dim3(gx, gy), 256, 0, st>>>(Q, ldq, n, j0, Qr, ldr);
    }
}

void launch_left_output(const double *Xw, int64_t ldw, int64_t n, int64_t m, const int32_t *dst,
                        int reverse, const int32_t *ew, const double *lrw, const double *liw,
                        double *X, int64_t ldx, int32_t *e, double *lr, double *li,
                        cudaStream_t st, const double *bw, double *bo) {
    if (n <= 0 || m <= 0) return;
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 16);
    for (int64_t c0 = 0; c0 < m; c0 += 65535) {
        const unsigned gy = (unsigned)std::min<int64_t>(m - c0, 65535);
        k_left_output<<<dim3(gx, gy), 256, 0, st>>>(Xw, ldw, n, c0, dst, reverse, ew, lrw, liw,
                                                    X, ldx, e, lr, li, bw, bo);
    }
}

}  // namespace evec
