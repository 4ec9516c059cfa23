// Algorithm 1 (preparation) on the GPU: factor every strip operator S^(j) A^(j)
// as a block-tridiagonal matrix along y, partitioned into P chunks separated by
// single separator rows (one level of nested dissection along y):
//
//   chunk p covers rows r0[p] .. r1[p]-1, separator p is row r1[p] (p < P-1).
//
// Per chunk (k_factor_chunk, one CTA per (chunk, strip), all in parallel):
//   S_{r0} = D_{r0},  S_k = D_k - C_k S_{k-1}^{-1} C_k   -> store Sinv_k = S_k^{-1}
//   bottom spike GB = A_p^{-1} E_last C_{r1}   (response to the separator below)
//   top spike    GT = A_p^{-1} E_first C_{r0}  (response to the separator above)
// so that the chunk solution is x_p = y_p - GT x_sep(p-1) - GB x_sep(p),
// y_p = A_p^{-1} b_p.
//
// Per strip (k_factor_reduced, one CTA per strip): the separators form a
// block-tridiagonal system with dense W x W blocks
//   T_q = D_s - C_s GB_q(last) - C_{s+1} GT_{q+1}(first),   s = r1[q]
//   L_q = -C_s GT_q(last),  U_q = -C_{s+1} GB_{q+1}(first)
// factored as R_q = T_q - L_q F_{q-1},  Rinv_q = R_q^{-1},  E_q = Rinv_q L_q,
// F_q = Rinv_q U_q, which the sweep runs as z_q = Rinv_q bhat_q - E_q z_{q-1},
// x_q = z_q - F_q x_{q+1}.
#include "common.cuh"
#include "strip_ops.cuh"
#include "internal.h"

namespace helm {

// Spikes are stored row-major (row c contiguous over columns a) so that the
// correction step can read only the rows it outputs; e is a column-major index.
__device__ __forceinline__ int trp(int e, int W) { return (e % W) * W + e / W; }

template <typename C>
__global__ void k_factor_chunk(Geom g, C* __restrict__ Sinv, C* __restrict__ GT, C* __restrict__ GB,
                               int* __restrict__ status) {
    const StripDev st = g.strips[blockIdx.y];
    const int p = blockIdx.x;
    const int W = st.W;
    const int r0 = g.r0[p], r1 = g.r1[p];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* M = reinterpret_cast<C*>(smem_raw);
    C* X = M + W * W;
    C* Y = X + W * W;
    C* dv = Y + W * W;          // W: diagonal coupling vector
    C* colk = dv + W;           // W: inverse scratch
    int* piv = reinterpret_cast<int*>(colk + W);
    double* red = reinterpret_cast<double*>(piv + ((W + 3) & ~3));

    C* SinvS = Sinv + st.fac;
    C* GTs = GT + st.fac;
    C* GBs = GB + st.fac;
    const int64_t bs = st.bs;

    // ---- block LU down the chunk
    for (int k = r0; k < r1; ++k) {
        build_diag_block(g, st, k, M);
        if (k > r0) {
            for (int c = threadIdx.x; c < W; c += blockDim.x)
                dv[c] = CT<C>::from(strip_coupling(g, st, k, c));
            __syncthreads();
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
                const int a = e % W, b = e / W;
                M[e] = csub(M[e], cmul(cmul(dv[a], X[e]), dv[b]));
            }
            __syncthreads();
        }
        if (!block_inverse(M, W, piv, colk, red)) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            return;
        }
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            SinvS[k * bs + e] = M[e];
            X[e] = M[e];
        }
        __syncthreads();
    }
    // X holds Sinv_{r1-1}

    // ---- bottom spike (driven by separator row r1 through C_{r1})
    if (p < g.P - 1) {
        for (int c = threadIdx.x; c < W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, r1, c));
        __syncthreads();
        // GB_last = Sinv_last diag(C_{r1})
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            const int b = e / W;
            Y[e] = cmul(X[e], dv[b]);
            GBs[(int64_t)(r1 - 1) * bs + trp(e, W)] = Y[e];
        }
        __syncthreads();
        // X <- Y (current spike block)
        block_copy(X, Y, W * W);
        for (int k = r1 - 2; k >= r0; --k) {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) M[e] = SinvS[(int64_t)k * bs + e];
            for (int c = threadIdx.x; c < W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, k + 1, c));
            __syncthreads();
            // GB_k = -Sinv_k diag(C_{k+1}) GB_{k+1}
            block_gemm_dscale(Y, M, dv, X, W, false, (typename CT<C>::R)-1);
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) GBs[(int64_t)k * bs + trp(e, W)] = Y[e];
            __syncthreads();
            block_copy(X, Y, W * W);
        }
    }

    // ---- top spike (driven by separator row r0-1 through C_{r0})
    if (p > 0) {
        // forward elimination of E_first C_{r0}: Z_{r0} = Sinv_{r0} diag(C_{r0}),
        // Z_k = -Sinv_k diag(C_k) Z_{k-1}; the Z_k are parked in GT.
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) M[e] = SinvS[(int64_t)r0 * bs + e];
        for (int c = threadIdx.x; c < W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, r0, c));
        __syncthreads();
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            const int b = e / W;
            X[e] = cmul(M[e], dv[b]);
            GTs[(int64_t)r0 * bs + trp(e, W)] = X[e];
        }
        __syncthreads();
        for (int k = r0 + 1; k < r1; ++k) {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) M[e] = SinvS[(int64_t)k * bs + e];
            for (int c = threadIdx.x; c < W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, k, c));
            __syncthreads();
            block_gemm_dscale(Y, M, dv, X, W, false, (typename CT<C>::R)-1);
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) GTs[(int64_t)k * bs + trp(e, W)] = Y[e];
            __syncthreads();
            block_copy(X, Y, W * W);
        }
        // back substitution: X_last = Z_last (already in GT and X);
        // X_k = Z_k - Sinv_k diag(C_{k+1}) X_{k+1}
        for (int k = r1 - 2; k >= r0; --k) {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
                M[e] = SinvS[(int64_t)k * bs + e];
                Y[e] = GTs[(int64_t)k * bs + trp(e, W)];
            }
            for (int c = threadIdx.x; c < W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, k + 1, c));
            __syncthreads();
            block_gemm_dscale(Y, M, dv, X, W, true, (typename CT<C>::R)-1);
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) GTs[(int64_t)k * bs + trp(e, W)] = Y[e];
            __syncthreads();
            block_copy(X, Y, W * W);
        }
    }
}

template <typename C>
__global__ void k_factor_reduced(Geom g, const C* __restrict__ GT, const C* __restrict__ GB,
                                 C* __restrict__ Rinv, C* __restrict__ E, C* __restrict__ F,
                                 int* __restrict__ status) {
    const StripDev st = g.strips[blockIdx.x];
    const int W = st.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* M = reinterpret_cast<C*>(smem_raw);
    C* X = M + W * W;
    C* Y = X + W * W;
    C* d0 = Y + W * W;          // C_s
    C* d1 = d0 + W;             // C_{s+1}
    C* colk = d1 + W;
    int* piv = reinterpret_cast<int*>(colk + W);
    double* red = reinterpret_cast<double*>(piv + ((W + 3) & ~3));
    const int64_t bs = st.bs;
    const C* GTs = GT + st.fac;
    const C* GBs = GB + st.fac;
    C* Rs = Rinv + st.red;
    C* Es = E + st.red;
    C* Fs = F + st.red;
    using R = typename CT<C>::R;

    for (int q = 0; q < g.P - 1; ++q) {
        const int s = g.r1[q];                 // separator row
        const int last_q = s - 1;              // last row of chunk q
        const int first_q1 = g.r0[q + 1];      // first row of chunk q+1 (= s+1)
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            d0[c] = CT<C>::from(strip_coupling(g, st, s, c));
            d1[c] = CT<C>::from(strip_coupling(g, st, s + 1, c));
        }
        build_diag_block(g, st, s, M);          // syncs
        // T = D_s - diag(C_s) GB_q(last) - diag(C_{s+1}) GT_{q+1}(first)
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            const int r = e % W;
            C t = M[e];
            t = csub(t, cmul(d0[r], GBs[(int64_t)last_q * bs + trp(e, W)]));
            t = csub(t, cmul(d1[r], GTs[(int64_t)first_q1 * bs + trp(e, W)]));
            M[e] = t;
        }
        __syncthreads();
        if (q >= 1) {
            // L_q = -diag(C_s) GT_q(last) -> X ; M -= L_q F_{q-1} (F_{q-1} in Y)
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
                const int r = e % W;
                X[e] = cneg(cmul(d0[r], GTs[(int64_t)last_q * bs + trp(e, W)]));
            }
            __syncthreads();
            block_gemm_dscale<C>(M, X, nullptr, Y, W, true, (R)-1);
        }
        if (!block_inverse(M, W, piv, colk, red)) {
            if (threadIdx.x == 0) atomicExch(status, 2);
            return;
        }
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) Rs[(int64_t)q * bs + e] = M[e];
        // E_q = Rinv_q L_q (zero for q = 0)
        if (q >= 1) {
            block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)1);
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) Es[(int64_t)q * bs + e] = Y[e];
        } else {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) Es[(int64_t)q * bs + e] = CT<C>::zero();
        }
        __syncthreads();
        // F_q = Rinv_q U_q, U_q = -diag(C_{s+1}) GB_{q+1}(first) (zero when chunk q+1 is last)
        if (q + 1 < g.P - 1) {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
                const int r = e % W;
                X[e] = cneg(cmul(d1[r], GBs[(int64_t)first_q1 * bs + trp(e, W)]));
            }
            __syncthreads();
            block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)1);
        } else {
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) Y[e] = CT<C>::zero();
            __syncthreads();
        }
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) Fs[(int64_t)q * bs + e] = Y[e];
        __syncthreads();
    }
}

size_t factor_smem_bytes(int Wmax, size_t esize) {
    return (size_t)3 * Wmax * Wmax * esize + (size_t)3 * Wmax * esize + (size_t)((Wmax + 3) & ~3) * 4 + 16;
}

template <typename C>
cudaError_t launch_factor(const Geom& g, int Wmax, void* Sinv, void* GT, void* GB, void* Rinv, void* E,
                          void* F, int* status, cudaStream_t s, KernelTimer* tm) {
    const size_t smem = factor_smem_bytes(Wmax, sizeof(C));
    cudaError_t err = cudaFuncSetAttribute(k_factor_chunk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_factor_reduced<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid(g.P, g.J);
    {
        TimedLaunch t(tm, "factor_chunk", s);
        k_factor_chunk<C><<<grid, 256, smem, s>>>(g, (C*)Sinv, (C*)GT, (C*)GB, status);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (g.P > 1) {
        TimedLaunch t(tm, "factor_reduced", s);
        k_factor_reduced<C><<<g.J, 256, smem, s>>>(g, (const C*)GT, (const C*)GB, (C*)Rinv, (C*)E, (C*)F,
                                                    status);
    }
    return cudaGetLastError();
}

template cudaError_t launch_factor<float2>(const Geom&, int, void*, void*, void*, void*, void*, void*, int*,
                                           cudaStream_t, KernelTimer*);
template cudaError_t launch_factor<double2>(const Geom&, int, void*, void*, void*, void*, void*, void*, int*,
                                            cudaStream_t, KernelTimer*);

}  // namespace helm
