// Algorithm 1 (preparation) on the GPU: factor every strip operator S^(j) A^(j)
// as a block-tridiagonal matrix along y, partitioned into P chunks separated by
// single separator rows (one level of nested dissection along y):
//
//   chunk p covers rows r0[p] .. r1[p]-1, separator p is row r1[p] (p < P-1).
//
// Every block-tridiagonal system (each chunk, and the separator system) is
// factored "twisted": eliminated from both ends toward a middle twist row, so
// that a solve runs its two halves concurrently and needs about m+1 dependent
// steps instead of 2m-1.  For a chunk with twist row t = r0 + (m-1)/2:
//   rows r0..t-1:   S_k = D_k - C_k S_{k-1}^{-1} C_k          (top down)
//   rows r1-1..t+1: S_k = D_k - C_{k+1} S_{k+1}^{-1} C_{k+1}  (bottom up)
//   row t:          S_t = D_t - C_t S_{t-1}^{-1} C_t - C_{t+1} S_{t+1}^{-1} C_{t+1}
// and Sinv_k = S_k^{-1} is stored for every row.  The chunk solve is
//   z_k = Sinv_k (b_k - C_k z_{k-1})        k < t
//   z_k = Sinv_k (b_k - C_{k+1} z_{k+1})    k > t
//   y_t = Sinv_t (b_t - C_t z_{t-1} - C_{t+1} z_{t+1})
//   y_k = z_k - Sinv_k C_{k+1} y_{k+1}      k < t (outward)
//   y_k = z_k - Sinv_k C_k y_{k-1}          k > t (outward).
// Spikes (k_factor_chunk): GB = A_p^{-1} E_last C_{r1} (response to the
// separator below) and GT = A_p^{-1} E_first C_{r0} (separator above), so that
// the chunk solution is x_p = y_p - GT x_sep(p-1) - GB x_sep(p).
//
// Separator system (k_factor_reduced, one CTA per strip), q = 0..Q-1, Q = P-1:
//   T_q = D_s - C_s GB_q(last) - C_{s+1} GT_{q+1}(first),   s = r1[q]
//   L_q = -C_s GT_q(last),  U_q = -C_{s+1} GB_{q+1}(first)
// twisted at tq = (Q-1)/2.  Stored per separator: Rinv_q, an "outer" coupling
// E_q (toward the ends) and an "inner" coupling F_q (toward the twist):
//   q < tq: R_q = T_q - L_q F_{q-1},  E_q = Rinv_q L_q,  F_q = Rinv_q U_q
//   q > tq: R_q = T_q - U_q F_{q+1},  E_q = Rinv_q U_q,  F_q = Rinv_q L_q
//   q = tq: R_q = T_q - L_q F_{q-1} - U_q F_{q+1},  E_q = Rinv_q L_q,  F_q = Rinv_q U_q
// and the separator solve is z_q = a_q - E_q z_{outer neighbour},
// x_tq = a_tq - E_tq z_{tq-1} - F_tq z_{tq+1}, x_q = z_q - F_q x_{inner neighbour},
// with a_q = Rinv_q bhat_q.
#include "common.cuh"
#include "strip_ops.cuh"
#include "internal.h"

namespace helm {

// Spikes are stored row-major (row c contiguous over columns a) so that the
// correction step can read only the rows it outputs; e is a column-major index.
__device__ __forceinline__ int trp(int e, int W) { return (e % W) * W + e / W; }

// shared (column-major W x W) <-> global sweep layout (row-major, ld, zero pad)
template <typename C>
__device__ void load_block(C* dst, const C* src, int W, int ld) {
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) dst[e] = src[(int64_t)(e % W) * ld + e / W];
}
template <typename C>
__device__ void store_block(C* dst, const C* src, int W, int ld) {
    for (int e = threadIdx.x; e < W * ld; e += blockDim.x) {
        const int r = e / ld, a = e % ld;
        dst[e] = a < W ? src[a * W + r] : CT<C>::zero();
    }
}
template <typename C>
__device__ void load_coupling(C* dv, const Geom& g, const StripDev& st, int k) {
    for (int c = threadIdx.x; c < st.W; c += blockDim.x) dv[c] = CT<C>::from(strip_coupling(g, st, k, c));
}
// M -= diag(d) X diag(d)
template <typename C>
__device__ void sub_congruence(C* M, const C* X, const C* d, int W) {
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        const int a = e % W, b = e / W;
        M[e] = csub(M[e], cmul(cmul(d[a], X[e]), d[b]));
    }
}

// Spike solve A_p Y = E_rs Rhs for the chunk [r0, r1) with twist t (rs = r0 or
// r1-1, Rhs = diag(C_{r0}) or diag(C_{r1}) given as the vector dr).  Y goes to
// OUT (global, row-major).  Z values of the elimination are parked in OUT.
// smem: M (Sinv), X (current), Y (scratch), dv (coupling vector).
template <typename C>
__device__ void spike_solve(const Geom& g, const StripDev& st, const C* SinvS, C* OUT, int r0, int r1, int t,
                            int rs, const C* dr, C* M, C* X, C* Y, C* dv) {
    using R = typename CT<C>::R;
    const int W = st.W;
    const int64_t bs = st.bs;
    auto store = [&](int k, const C* src) {
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) OUT[(int64_t)k * bs + trp(e, W)] = src[e];
    };
    auto fetch = [&](C* dst, int k) {
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) dst[e] = OUT[(int64_t)k * bs + trp(e, W)];
    };
    // X <- Sinv_rs diag(dr): the eliminated block at row rs
    load_block(M, SinvS + (int64_t)rs * bs, W, st.ld);
    __syncthreads();
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) X[e] = cmul(M[e], dr[e / W]);
    __syncthreads();
    if (rs != t) {
        store(rs, X);
        const int dir = rs < t ? 1 : -1;   // elimination runs toward the twist
        for (int k = rs + dir; k != t; k += dir) {
            load_block(M, SinvS + (int64_t)k * bs, W, st.ld);
            load_coupling(dv, g, st, dir > 0 ? k : k + 1);   // coupling to the previous row
            __syncthreads();
            block_gemm_dscale(Y, M, dv, X, W, false, (R)-1);   // z_k = -Sinv_k C z_prev
            store(k, Y);
            __syncthreads();
            block_copy(X, Y, W * W);
        }
        // twist row: y_t = Sinv_t (-C z_{t-dir})
        load_block(M, SinvS + (int64_t)t * bs, W, st.ld);
        load_coupling(dv, g, st, dir > 0 ? t : t + 1);
        __syncthreads();
        block_gemm_dscale(Y, M, dv, X, W, false, (R)-1);
        block_copy(X, Y, W * W);
    }
    store(t, X);                               // X = y_t
    __syncthreads();
    // outward back substitution on both sides; Y_k = z_k - Sinv_k C y_inner
    for (int side = 0; side < 2; ++side) {
        const int dir = side == 0 ? -1 : 1;      // -1: rows t-1..r0, +1: rows t+1..r1-1
        fetch(X, t);                             // y_t
        __syncthreads();
        for (int k = t + dir; k >= r0 && k < r1; k += dir) {
            load_block(M, SinvS + (int64_t)k * bs, W, st.ld);
            load_coupling(dv, g, st, dir < 0 ? k + 1 : k);   // coupling to the inner row
            const bool has_z = (rs < t) ? (dir < 0 && k >= rs) : (rs > t && dir > 0 && k <= rs);
            if (has_z) fetch(Y, k);
            else for (int e = threadIdx.x; e < W * W; e += blockDim.x) Y[e] = CT<C>::zero();
            __syncthreads();
            block_gemm_dscale(Y, M, dv, X, W, true, (R)-1);
            store(k, Y);
            __syncthreads();
            block_copy(X, Y, W * W);
        }
    }
}

template <typename C>
__global__ void k_factor_chunk(Geom g, C* __restrict__ Sinv, C* __restrict__ GT, C* __restrict__ GB,
                               int* __restrict__ status) {
    const StripDev st = g.strips[blockIdx.y];
    const int p = blockIdx.x;
    const int W = st.W;
    const int r0 = g.r0[p], r1 = g.r1[p];
    const int t = r0 + (r1 - r0 - 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* M = reinterpret_cast<C*>(smem_raw);
    C* X = M + W * W;
    C* Y = X + W * W;
    C* dv = Y + W * W;          // W: diagonal coupling vector
    C* colk = dv + W;           // W: inverse scratch
    int* piv = reinterpret_cast<int*>(colk + W);
    double* red = reinterpret_cast<double*>(piv + ((W + 3) & ~3));
    C* SinvS = Sinv + st.fac;
    const int64_t bs = st.bs;

    auto finish_row = [&](int k) -> bool {
        if (!block_inverse(M, W, piv, colk, red)) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            return false;
        }
        store_block(SinvS + (int64_t)k * bs, M, W, st.ld);
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) X[e] = M[e];
        __syncthreads();
        return true;
    };
    // ---- top-down rows r0 .. t-1
    for (int k = r0; k < t; ++k) {
        build_diag_block(g, st, k, M);
        if (k > r0) {
            load_coupling(dv, g, st, k);
            __syncthreads();
            sub_congruence(M, X, dv, W);
            __syncthreads();
        }
        if (!finish_row(k)) return;
    }
    // ---- bottom-up rows r1-1 .. t+1
    for (int k = r1 - 1; k > t; --k) {
        build_diag_block(g, st, k, M);
        if (k < r1 - 1) {
            load_coupling(dv, g, st, k + 1);
            __syncthreads();
            sub_congruence(M, X, dv, W);
            __syncthreads();
        }
        if (!finish_row(k)) return;
    }
    // ---- twist row
    build_diag_block(g, st, t, M);
    if (t > r0) {
        load_block(X, SinvS + (int64_t)(t - 1) * bs, W, st.ld);
        load_coupling(dv, g, st, t);
        __syncthreads();
        sub_congruence(M, X, dv, W);
        __syncthreads();
    }
    if (t < r1 - 1) {
        load_block(X, SinvS + (int64_t)(t + 1) * bs, W, st.ld);
        load_coupling(dv, g, st, t + 1);
        __syncthreads();
        sub_congruence(M, X, dv, W);
        __syncthreads();
    }
    if (!finish_row(t)) return;

    // ---- spikes
    C* dr = colk;   // right-hand-side coupling (colk is free outside the inverse)
    if (p < g.P - 1) {   // bottom spike, driven by separator row r1
        load_coupling(dr, g, st, r1);
        __syncthreads();
        spike_solve(g, st, SinvS, GB + st.fac, r0, r1, t, r1 - 1, dr, M, X, Y, dv);
        __syncthreads();
    }
    if (p > 0) {         // top spike, driven by separator row r0-1
        load_coupling(dr, g, st, r0);
        __syncthreads();
        spike_solve(g, st, SinvS, GT + st.fac, r0, r1, t, r0, dr, M, X, Y, dv);
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
    const int Q = g.P - 1;
    const int tq = (Q - 1) / 2;

    // M <- T_q; leaves C_s in d0 and C_{s+1} in d1
    auto build_T = [&](int q) {
        const int s = g.r1[q];
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
            d0[c] = CT<C>::from(strip_coupling(g, st, s, c));
            d1[c] = CT<C>::from(strip_coupling(g, st, s + 1, c));
        }
        build_diag_block(g, st, s, M);
        const int last_q = s - 1, first_q1 = g.r0[q + 1];
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            const int r = e % W;
            C tt = M[e];
            tt = csub(tt, cmul(d0[r], GBs[(int64_t)last_q * bs + trp(e, W)]));
            tt = csub(tt, cmul(d1[r], GTs[(int64_t)first_q1 * bs + trp(e, W)]));
            M[e] = tt;
        }
        __syncthreads();
    };
    // X <- L_q = -C_s GT_q(last)   (q >= 1)
    auto build_L = [&](int q, C* D) {
        const int last_q = g.r1[q] - 1;
        for (int e = threadIdx.x; e < W * W; e += blockDim.x)
            D[e] = cneg(cmul(d0[e % W], GTs[(int64_t)last_q * bs + trp(e, W)]));
        __syncthreads();
    };
    // D <- U_q = -C_{s+1} GB_{q+1}(first)   (q <= Q-2)
    auto build_U = [&](int q, C* D) {
        const int first_q1 = g.r0[q + 1];
        for (int e = threadIdx.x; e < W * W; e += blockDim.x)
            D[e] = cneg(cmul(d1[e % W], GBs[(int64_t)first_q1 * bs + trp(e, W)]));
        __syncthreads();
    };
    auto invert_store = [&](int q) -> bool {
        if (!block_inverse(M, W, piv, colk, red)) {
            if (threadIdx.x == 0) atomicExch(status, 2);
            return false;
        }
        store_block(Rs + (int64_t)q * bs, M, W, st.ld);
        __syncthreads();
        return true;
    };
    // out = Rinv_q D  -> global slot
    auto store_prod = [&](C* slot, const C* D) {
        block_gemm_dscale<C>(Y, M, nullptr, D, W, false, (R)1);
        store_block(slot, Y, W, st.ld);
        __syncthreads();
    };
    auto zero_slot = [&](C* slot) {
        for (int e = threadIdx.x; e < W * st.ld; e += blockDim.x) slot[e] = CT<C>::zero();
        __syncthreads();
    };
    auto inner = [&](int q) -> const C* { return Fs + (int64_t)q * bs; };   // stored F of a neighbour
    // T -= D * F_nb with D built in X and F_nb read into Y
    auto sub_coupled = [&](const C* Fnb) {
        load_block(Y, Fnb, W, st.ld);
        __syncthreads();
        block_gemm_dscale<C>(M, X, nullptr, Y, W, true, (R)-1);
    };
    // ---- top-down q = 0 .. tq-1
    for (int q = 0; q < tq; ++q) {
        build_T(q);
        if (q >= 1) { build_L(q, X); sub_coupled(inner(q - 1)); }
        if (!invert_store(q)) return;
        if (q >= 1) { build_L(q, X); store_prod(Es + (int64_t)q * bs, X); }
        else zero_slot(Es + (int64_t)q * bs);
        build_U(q, X);
        store_prod(Fs + (int64_t)q * bs, X);
    }
    // ---- bottom-up q = Q-1 .. tq+1
    for (int q = Q - 1; q > tq; --q) {
        build_T(q);
        if (q <= Q - 2) { build_U(q, X); sub_coupled(inner(q + 1)); }
        if (!invert_store(q)) return;
        if (q <= Q - 2) { build_U(q, X); store_prod(Es + (int64_t)q * bs, X); }
        else zero_slot(Es + (int64_t)q * bs);
        build_L(q, X);
        store_prod(Fs + (int64_t)q * bs, X);
    }
    // ---- twist q = tq (its F slot is written last: the neighbours' F are read first)
    if (Q >= 1) {
        const int q = tq;
        build_T(q);
        if (q >= 1) { build_L(q, X); sub_coupled(inner(q - 1)); }
        if (q <= Q - 2) { build_U(q, X); sub_coupled(inner(q + 1)); }
        if (!invert_store(q)) return;
        if (q >= 1) { build_L(q, X); store_prod(Es + (int64_t)q * bs, X); }
        else zero_slot(Es + (int64_t)q * bs);
        if (q <= Q - 2) { build_U(q, X); store_prod(Fs + (int64_t)q * bs, X); }
        else zero_slot(Fs + (int64_t)q * bs);
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
