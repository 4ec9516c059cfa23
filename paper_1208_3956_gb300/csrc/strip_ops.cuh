// Block-row coefficients of the symmetrised strip operator S^(j) A^(j) and the
// block-level dense kernels (Gauss-Jordan inverse, products) shared by the
// factorisation kernels.
//
// Ordering: the strip's unknowns are grouped by grid row y = k (block k holds
// the W columns of the strip).  S^(j) A^(j) is then block tridiagonal:
//   diagonal block D_k  = tridiagonal W x W (x-part of Section 2.2 plus the
//                         y-diagonal and -S k^2),
//   coupling   C_k      = diagonal, couples rows k-1 and k,
//                         C_k(c) = -s_x(c) alpha_y(y_{k-1/2}) / h^2.
// Symmetrised entries (row (c,k) of A times s_x(c) s_y(k), s = 1/alpha):
//   D_k(c,c)   = s_y(k)[a_x(c+1/2) + a_x(c-1/2)]/h^2 + s_x(c)[a_y(k+1/2) + a_y(k-1/2)]/h^2
//                - s_x(c) s_y(k) k^2(c,k)
//   D_k(c,c+1) = D_k(c+1,c) = -s_y(k) a_x(c+1/2)/h^2
// With Robin transmission the strips carry no added layers and the diagonal of an
// internal boundary column gains s_x s_y (a/b)/h^2 (Geom::rab).
#pragma once

#include "common.cuh"

namespace helm {

__device__ __forceinline__ double2 strip_ax_int(const Geom& g, const StripDev& st, int c) {
    return g.stab[st.tab + c];
}
__device__ __forceinline__ double2 strip_ax_half(const Geom& g, const StripDev& st, int m) {
    return g.stab[st.tab + st.W + m];   // alpha at strip half point m - 1/2
}
__device__ __forceinline__ int strip_k2_col(const StripDev& st, int c) {
    return imin(imax(st.lo - st.lpml + c, st.lo), st.hi);
}
__device__ __forceinline__ double2 strip_sx(const Geom& g, const StripDev& st, int c) {
    return cinv(strip_ax_int(g, st, c));
}
__device__ __forceinline__ double2 glob_sy(const Geom& g, int k) { return cinv(g.gy_int[k]); }

// C_k(c): coupling between rows k-1 and k (k >= 1), symmetric form.
__device__ __forceinline__ double2 strip_coupling(const Geom& g, const StripDev& st, int k, int c) {
    return cscale(cmul(strip_sx(g, st, c), g.gy_half[k]), -g.inv_h2);
}

// diagonal and super-diagonal entries of D_k
__device__ __forceinline__ double2 strip_diag(const Geom& g, const StripDev& st, int k, int c) {
    double2 sx = strip_sx(g, st, c);
    double2 sy = glob_sy(g, k);
    double2 xs = cadd(strip_ax_half(g, st, c + 1), strip_ax_half(g, st, c));
    double2 ys = cadd(g.gy_half[k + 1], g.gy_half[k]);
    double2 d = cscale(cadd(cmul(sy, xs), cmul(sx, ys)), g.inv_h2);
    double k2 = g.k2[(int64_t)k * g.Nx + strip_k2_col(st, c)];
    d = csub(d, cscale(cmul(sx, sy), k2));
    if (g.rab) {
        // Robin rows (Section 4.4): the ghost value beyond an internal boundary column,
        // eliminated through a u_in + b u_ghost = data, adds (a/b)/h^2 to the diagonal
        if (c == 0 && st.j > 0) d = cadd(d, cscale(cmul(cmul(sx, sy), g.rab[(int64_t)st.j * g.Ny + k]), g.inv_h2));
        if (c == st.W - 1 && st.j < g.J - 1)
            d = cadd(d, cscale(cmul(cmul(sx, sy), g.rab[(int64_t)(st.j + 1) * g.Ny + k]), g.inv_h2));
    }
    return d;
}
__device__ __forceinline__ double2 strip_offdiag(const Geom& g, const StripDev& st, int k, int c) {
    // entry (c, c+1) = (c+1, c)
    return cscale(cmul(glob_sy(g, k), strip_ax_half(g, st, c + 1)), -g.inv_h2);
}

// M <- D_k, column-major with leading dimension W.  Whole block participates.
template <typename C>
__device__ void build_diag_block(const Geom& g, const StripDev& st, int k, C* M) {
    const int W = st.W;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) M[e] = CT<C>::zero();
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        M[c * W + c] = CT<C>::from(strip_diag(g, st, k, c));
        if (c + 1 < W) {
            C o = CT<C>::from(strip_offdiag(g, st, k, c));
            M[(c + 1) * W + c] = o;
            M[c * W + c + 1] = o;
        }
    }
    __syncthreads();
}

// In-place Gauss-Jordan inverse with partial (row) pivoting of the W x W
// column-major matrix A in shared memory.  piv: int[W], colk: C[W], red: 2
// doubles of scratch.  Returns false (uniformly) on a zero or non-finite pivot.
template <typename C>
__device__ bool block_inverse(C* A, int n, int* piv, C* colk, double* red) {
    using R = typename CT<C>::R;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            R best = (R)-1;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                R v = cabs2(A[k * n + i]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                R ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) { piv[k] = bi; red[0] = (double)best; }
        }
        __syncthreads();
        const double pmag = red[0];
        if (!(pmag > 0.0) || !isfinite(pmag)) return false;   // uniform across the block
        const int p = piv[k];
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                C t = A[j * n + k]; A[j * n + k] = A[j * n + p]; A[j * n + p] = t;
            }
        }
        __syncthreads();
        const C inv = cinv(A[k * n + k]);
        for (int i = tid; i < n; i += nt) colk[i] = (i == k) ? CT<C>::zero() : A[k * n + i];
        __syncthreads();
        for (int j = tid; j < n; j += nt) A[j * n + k] = (j == k) ? inv : cmul(A[j * n + k], inv);
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            const int i = e % n, j = e / n;
            if (i == k) continue;
            C a = (j == k) ? CT<C>::zero() : A[e];
            A[e] = csub(a, cmul(colk[i], A[j * n + k]));
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k) {
            for (int i = tid; i < n; i += nt) {
                C t = A[k * n + i]; A[k * n + i] = A[p * n + i]; A[p * n + i] = t;
            }
        }
        __syncthreads();
    }
    return true;
}

// Out(r,c) = beta*Out(r,c) + sgn * sum_a A(r,a) d(a) B(a,c)   (column-major, W x W;
// d: optional diagonal scaling between the factors; Out may alias neither A nor B).
template <typename C>
__device__ void block_gemm_dscale(C* Out, const C* A, const C* d, const C* B, int n, bool accumulate,
                                  typename CT<C>::R sgn) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e % n, c = e / n;
        C acc = CT<C>::zero();
        if (d) {
            for (int a = 0; a < n; ++a) acc = cfma(A[a * n + r], cmul(d[a], B[c * n + a]), acc);
        } else {
            for (int a = 0; a < n; ++a) acc = cfma(A[a * n + r], B[c * n + a], acc);
        }
        acc = cscale(acc, sgn);
        Out[e] = accumulate ? cadd(Out[e], acc) : acc;
    }
    __syncthreads();
}

template <typename C>
__device__ void block_copy(C* dst, const C* src, int count) {
    for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = src[e];
    __syncthreads();
}

}  // namespace helm
