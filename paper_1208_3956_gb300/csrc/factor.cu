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
// Separator system (k_factor_sep, one CTA per strip), q = 0..Q-1, Q = P-1, solved
// in groups (a second level of nested dissection, see k_factor_sep):
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

// Spikes are stored row-major (row c contiguous over columns a, row length
// spld(W)) so that the correction step can stage only the rows it outputs; e is
// a column-major index.
__device__ __forceinline__ int trp(int e, int W) { return (e % W) * spld(W) + e / W; }

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

// Twisted LU of a block-tridiagonal system with dense couplings, elements
// i = 0..n-1 stored at separator slots sl(i): bT(i) builds the diagonal block
// into M, bL(i, D) / bU(i, D) build the couplings to i-1 / i+1 into D (they may
// use Y and Z as scratch but not M).  Stores Rinv, the outer coupling E and the
// inner coupling F of every element (see the file header).  Shared buffers:
// M, X, Y, Z (column-major W x W).
template <typename C, typename SL, typename BT_, typename BL, typename BU>
__device__ bool twisted_lu(const StripDev& st, int n, SL sl, BT_ bT, BL bL, BU bU, C* Rp, C* Ep, C* Fp, C* M,
                           C* X, C* Y, int* piv, C* colk, double* red, int* status) {
    using R = typename CT<C>::R;
    const int W = st.W;
    const int64_t bs = st.bs;
    auto slot = [&](C* pool, int i) { return pool + (int64_t)sl(i) * bs; };
    auto sub_nb = [&](C* Fpool, int inb) {   // M -= X F_nb
        load_block(Y, slot(Fpool, inb), W, st.ld);
        __syncthreads();
        block_gemm_dscale<C>(M, X, nullptr, Y, W, true, (R)-1);
    };
    auto inv_store = [&](int i) -> bool {
        if (!block_inverse(M, W, piv, colk, red)) {
            if (threadIdx.x == 0) atomicExch(status, 2);
            return false;
        }
        store_block(slot(Rp, i), M, W, st.ld);
        __syncthreads();
        return true;
    };
    auto prod_store = [&](C* dst) {   // dst = M X (M = Rinv)
        block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)1);
        store_block(dst, Y, W, st.ld);
        __syncthreads();
    };
    auto zero_store = [&](C* dst) {
        for (int e = threadIdx.x; e < W * st.ld; e += blockDim.x) dst[e] = CT<C>::zero();
        __syncthreads();
    };
    const int tq = (n - 1) / 2;
    for (int i = 0; i < tq; ++i) {                   // top down
        bT(i);
        if (i >= 1) { bL(i, X); sub_nb(Fp, i - 1); }
        if (!inv_store(i)) return false;
        if (i >= 1) { bL(i, X); prod_store(slot(Ep, i)); } else zero_store(slot(Ep, i));
        bU(i, X);
        prod_store(slot(Fp, i));
    }
    for (int i = n - 1; i > tq; --i) {               // bottom up
        bT(i);
        if (i <= n - 2) { bU(i, X); sub_nb(Fp, i + 1); }
        if (!inv_store(i)) return false;
        if (i <= n - 2) { bU(i, X); prod_store(slot(Ep, i)); } else zero_store(slot(Ep, i));
        bL(i, X);
        prod_store(slot(Fp, i));
    }
    {                                                // twist
        const int i = tq;
        bT(i);
        if (i >= 1) { bL(i, X); sub_nb(Fp, i - 1); }
        if (i <= n - 2) { bU(i, X); sub_nb(Fp, i + 1); }
        if (!inv_store(i)) return false;
        if (i >= 1) { bL(i, X); prod_store(slot(Ep, i)); } else zero_store(slot(Ep, i));
        if (i <= n - 2) { bU(i, X); prod_store(slot(Fp, i)); } else zero_store(slot(Fp, i));
    }
    return true;
}

template <typename C>
struct SepPools {
    C* Rinv;   // per separator slot, sweep layout
    C* E;
    C* F;
    C* GT2;    // group spikes, row-major W x W
    C* GB2;
    C* P2L;    // level-2 right-hand-side products Rinv2 L, Rinv2 U (sweep layout)
    C* P2U;
    C* Q2L;    // level-2 contributions of a group separator's right-hand side (sweep layout)
    C* Q2U;
};

// Separator system of every strip (one CTA per strip): twisted LU of each group,
// the group spikes, and (G > 1) the level-2 system and its products.
template <typename C>
__global__ void k_factor_sep(Geom g, const C* __restrict__ GT, const C* __restrict__ GB, SepPools<C> pl,
                             int* __restrict__ status) {
    const StripDev st = g.strips[blockIdx.x];
    const int W = st.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* M = reinterpret_cast<C*>(smem_raw);
    C* X = M + W * W;
    C* Y = X + W * W;
    C* Z = g.G > 1 ? Y + W * W : nullptr;   // level-2 scratch, only with groups
    C* colk = Y + (g.G > 1 ? 2 : 1) * W * W + W;
    int* piv = reinterpret_cast<int*>(colk + W);
    double* red = reinterpret_cast<double*>(piv + ((W + 3) & ~3));
    using R = typename CT<C>::R;
    const int64_t bs = st.bs;
    const C* GTs = GT + st.fac;
    const C* GBs = GB + st.fac;
    SepPools<C> P = pl;
    P.Rinv += st.red; P.E += st.red; P.F += st.red; P.GT2 += st.red; P.GB2 += st.red; P.P2L += st.red;
    P.P2U += st.red;
    if (P.Q2L) { P.Q2L += st.red; P.Q2U += st.red; }
    const int G = g.G;

    // ---- level-1 blocks of separator q (row s = r1[q])
    auto build_T1 = [&](int q) {   // M <- T_q = D_s - C_s GB_q(last) - C_{s+1} GT_{q+1}(first)
        const int s = g.r1[q];
        build_diag_block(g, st, s, M);
        const int last_q = s - 1, first_q1 = g.r0[q + 1];
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
            const int r = e % W;
            C tt = M[e];
            tt = csub(tt, cmul(CT<C>::from(strip_coupling(g, st, s, r)), GBs[(int64_t)last_q * bs + trp(e, W)]));
            tt = csub(tt, cmul(CT<C>::from(strip_coupling(g, st, s + 1, r)), GTs[(int64_t)first_q1 * bs + trp(e, W)]));
            M[e] = tt;
        }
        __syncthreads();
    };
    auto build_L1 = [&](int q, C* D) {   // L_q = -C_s GT_q(last)
        const int s = g.r1[q];
        for (int e = threadIdx.x; e < W * W; e += blockDim.x)
            D[e] = cneg(cmul(CT<C>::from(strip_coupling(g, st, s, e % W)), GTs[(int64_t)(s - 1) * bs + trp(e, W)]));
        __syncthreads();
    };
    auto build_U1 = [&](int q, C* D) {   // U_q = -C_{s+1} GB_{q+1}(first)
        const int s = g.r1[q];
        const int first_q1 = g.r0[q + 1];
        for (int e = threadIdx.x; e < W * W; e += blockDim.x)
            D[e] = cneg(cmul(CT<C>::from(strip_coupling(g, st, s + 1, e % W)), GBs[(int64_t)first_q1 * bs + trp(e, W)]));
        __syncthreads();
    };

    // ---- groups: twisted LU of each group's separators
    for (int gi = 0; gi < G; ++gi) {
        const int q0 = g.gq0[gi], n = g.gq1[gi] - q0;
        auto sl = [&](int i) { return q0 + i; };
        if (!twisted_lu<C>(st, n, sl, [&](int i) { build_T1(q0 + i); },
                           [&](int i, C* D) { build_L1(q0 + i, D); }, [&](int i, C* D) { build_U1(q0 + i, D); },
                           P.Rinv, P.E, P.F, M, X, Y, piv, colk, red, status))
            return;
    }
    if (G == 1) return;

    // ---- group spikes: response of group gi to the level-2 separator above
    // (right-hand side L_{q0} at its first element) and below (U_{q1-1} at its last)
    auto rowmajor_store = [&](C* dst, const C* src) {
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) dst[trp(e, W)] = src[e];
    };
    auto rowmajor_load = [&](C* dst, const C* src) {
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) dst[e] = src[trp(e, W)];
    };
    for (int gi = 0; gi < G; ++gi) {
        const int q0 = g.gq0[gi], q1 = g.gq1[gi], n = q1 - q0, tq = (n - 1) / 2;
        for (int side = 0; side < 2; ++side) {
            const bool top = side == 0;
            if (top && gi == 0) continue;
            if (!top && gi == G - 1) continue;
            C* OUT = top ? P.GT2 : P.GB2;
            auto out = [&](int i) { return OUT + (int64_t)(q0 + i) * bs; };
            const int rs = top ? 0 : n - 1;
            // X <- Rinv_rs B, B = L_{q0} (top) or U_{q1-1} (bottom)
            if (top) build_L1(q0, Z); else build_U1(q1 - 1, Z);
            load_block(M, P.Rinv + (int64_t)(q0 + rs) * bs, W, st.ld);
            __syncthreads();
            block_gemm_dscale<C>(X, M, nullptr, Z, W, false, (R)1);
            if (rs != tq) {
                rowmajor_store(out(rs), X);
                const int dir = rs < tq ? 1 : -1;
                for (int i = rs + dir; i != tq; i += dir) {   // z_i = -E_i z_prev
                    load_block(M, P.E + (int64_t)(q0 + i) * bs, W, st.ld);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)-1);
                    rowmajor_store(out(i), Y);
                    __syncthreads();
                    block_copy(X, Y, W * W);
                }
                // twist: x_t = -E_t z_{t-1} (from above) or -F_t z_{t+1} (from below)
                load_block(M, (dir > 0 ? P.E : P.F) + (int64_t)(q0 + tq) * bs, W, st.ld);
                __syncthreads();
                block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)-1);
                block_copy(X, Y, W * W);
            }
            rowmajor_store(out(tq), X);
            __syncthreads();
            for (int sd = 0; sd < 2; ++sd) {   // outward: x_i = z_i - F_i x_inner
                const int dir = sd == 0 ? -1 : 1;
                rowmajor_load(X, out(tq));
                __syncthreads();
                for (int i = tq + dir; i >= 0 && i < n; i += dir) {
                    load_block(M, P.F + (int64_t)(q0 + i) * bs, W, st.ld);
                    const bool has_z = top ? (dir < 0 && i >= rs) : (dir > 0 && i <= rs);
                    if (has_z) rowmajor_load(Y, out(i));
                    else for (int e = threadIdx.x; e < W * W; e += blockDim.x) Y[e] = CT<C>::zero();
                    __syncthreads();
                    block_gemm_dscale<C>(Y, M, nullptr, X, W, true, (R)-1);
                    rowmajor_store(out(i), Y);
                    __syncthreads();
                    block_copy(X, Y, W * W);
                }
            }
        }
    }

    // ---- level-2 system over r = 0..G-2 (separator sigma_r = gq1[r])
    auto sig = [&](int r) { return g.gq1[r]; };
    auto bT2 = [&](int r) {   // T_s - L_s GB2_r(last) - U_s GT2_{r+1}(first)
        const int q = sig(r);
        build_T1(q);
        build_L1(q, Z);
        rowmajor_load(Y, P.GB2 + (int64_t)(q - 1) * bs);
        __syncthreads();
        block_gemm_dscale<C>(M, Z, nullptr, Y, W, true, (R)-1);
        build_U1(q, Z);
        rowmajor_load(Y, P.GT2 + (int64_t)g.gq0[r + 1] * bs);
        __syncthreads();
        block_gemm_dscale<C>(M, Z, nullptr, Y, W, true, (R)-1);
    };
    auto bL2 = [&](int r, C* D) {   // -L_s GT2_r(last)
        const int q = sig(r);
        build_L1(q, Z);
        rowmajor_load(Y, P.GT2 + (int64_t)(q - 1) * bs);
        __syncthreads();
        block_gemm_dscale<C>(D, Z, nullptr, Y, W, false, (R)-1);
    };
    auto bU2 = [&](int r, C* D) {   // -U_s GB2_{r+1}(first)
        const int q = sig(r);
        build_U1(q, Z);
        rowmajor_load(Y, P.GB2 + (int64_t)g.gq0[r + 1] * bs);
        __syncthreads();
        block_gemm_dscale<C>(D, Z, nullptr, Y, W, false, (R)-1);
    };
    if (!twisted_lu<C>(st, G - 1, sig, bT2, bL2, bU2, P.Rinv, P.E, P.F, M, X, Y, piv, colk, red, status)) return;
    // level-2 right-hand-side products: P2L_r = Rinv2_r L_s, P2U_r = Rinv2_r U_s
    for (int r = 0; r < G - 1; ++r) {
        const int q = sig(r);
        load_block(M, P.Rinv + (int64_t)q * bs, W, st.ld);
        build_L1(q, X);
        block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)1);
        store_block(P.P2L + (int64_t)q * bs, Y, W, st.ld);
        build_U1(q, X);
        __syncthreads();
        block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)1);
        store_block(P.P2U + (int64_t)q * bs, Y, W, st.ld);
        __syncthreads();
    }
    if (!P.Q2L) return;

    // ---- level-2 contributions of the group separators.  A group's part of a level-2
    // right-hand side is -P2L y(last) (to the level-2 separator below it) or -P2U y(first)
    // (above), and the group solution's end values are linear in the group's right-hand sides
    // a_i = Rinv_i bhat_i: y(last) = sum_i K_i a_i, y(first) = sum_i K'_i a_i.  The K blocks
    // follow from the twisted solve's recurrences run backwards (the derivative of its last or
    // first output with respect to every intermediate):
    //   y(last):  G_{n-1} = I, G_{j-1} = -G_j F_j (j > tq); K_tq = G_tq;
    //             K_{tq-1} = -G_tq E_tq, K_{j-1} = -K_j E_j (j < tq);
    //             K_{tq+1} = G_{tq+1} - G_tq F_tq, K_j = G_j - K_{j-1} E_{j-1} (j > tq + 1)
    //   y(first): G'_0 = I, G'_{j+1} = -G'_j F_j (j < tq); K'_tq = G'_tq;
    //             K'_{tq+1} = -G'_tq F_tq, K'_{j+1} = -K'_j E_j (j > tq);
    //             K'_{tq-1} = G'_{tq-1} - G'_tq E_tq, K'_{j-1} = G'_{j-1} - K'_j E_j (j < tq - 1)
    // Stored per separator: Q2L_i = -P2L K_i, Q2U_i = -P2U K'_i, so that every chunk adds its
    // share of the level-2 right-hand sides from its own separator parts.
    const C one = CT<C>::from(make_double2(1.0, 0.0));
    auto ident = [&](C* D) {
        for (int e = threadIdx.x; e < W * W; e += blockDim.x) D[e] = (e % W == e / W) ? one : CT<C>::zero();
        __syncthreads();
    };
    for (int gi = 0; gi < G; ++gi) {
        const int q0 = g.gq0[gi], q1 = g.gq1[gi], n = q1 - q0, tq = (n - 1) / 2;
        for (int side = 0; side < 2; ++side) {
            const bool last = side == 0;   // y(last): level-2 separator below; y(first): above
            if (last && gi == G - 1) continue;
            if (!last && gi == 0) continue;
            C* OUT = last ? P.Q2L : P.Q2U;
            auto slot = [&](int i) { return OUT + (int64_t)(q0 + i) * bs; };
            auto put = [&](int i, const C* src) {
                rowmajor_store(slot(i), src);
                __syncthreads();
            };
            auto get = [&](C* dst, int i) { rowmajor_load(dst, slot(i)); };
            auto blk = [&](C* dst, const C* pool, int i) { load_block(dst, pool + (int64_t)(q0 + i) * bs, W, st.ld); };
            if (last) {
                ident(X);
                put(n - 1, X);
                for (int j = n - 1; j > tq; --j) {   // G_{j-1} = -G_j F_j
                    blk(M, P.F, j);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, X, nullptr, M, W, false, (R)-1);
                    block_copy(X, Y, W * W);
                    put(j - 1, X);
                }
                block_copy(Z, X, W * W);             // G_tq = K_tq
                for (int j = tq; j >= 1; --j) {      // K_{j-1} = -K_j E_j (K_tq = G_tq)
                    blk(M, P.E, j);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, Z, nullptr, M, W, false, (R)-1);
                    block_copy(Z, Y, W * W);
                    put(j - 1, Z);
                }
                if (n - 1 > tq) {                    // K_{tq+1} = G_{tq+1} - G_tq F_tq
                    get(Z, tq);
                    blk(M, P.F, tq);
                    get(Y, tq + 1);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, Z, nullptr, M, W, true, (R)-1);
                    put(tq + 1, Y);
                    block_copy(Z, Y, W * W);
                    for (int j = tq + 2; j < n; ++j) {   // K_j = G_j - K_{j-1} E_{j-1}
                        blk(M, P.E, j - 1);
                        get(Y, j);
                        __syncthreads();
                        block_gemm_dscale<C>(Y, Z, nullptr, M, W, true, (R)-1);
                        put(j, Y);
                        block_copy(Z, Y, W * W);
                    }
                }
            } else {
                ident(X);
                put(0, X);
                for (int j = 0; j < tq; ++j) {       // G'_{j+1} = -G'_j F_j
                    blk(M, P.F, j);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, X, nullptr, M, W, false, (R)-1);
                    block_copy(X, Y, W * W);
                    put(j + 1, X);
                }
                if (n - 1 > tq) {                    // K'_{tq+1} = -G'_tq F_tq, K'_{j+1} = -K'_j E_j
                    blk(M, P.F, tq);
                    __syncthreads();
                    block_gemm_dscale<C>(Z, X, nullptr, M, W, false, (R)-1);
                    put(tq + 1, Z);
                    for (int j = tq + 1; j + 1 < n; ++j) {
                        blk(M, P.E, j);
                        __syncthreads();
                        block_gemm_dscale<C>(Y, Z, nullptr, M, W, false, (R)-1);
                        block_copy(Z, Y, W * W);
                        put(j + 1, Z);
                    }
                }
                if (tq >= 1) {                       // K'_{tq-1} = G'_{tq-1} - G'_tq E_tq
                    block_copy(Z, X, W * W);
                    blk(M, P.E, tq);
                    get(Y, tq - 1);
                    __syncthreads();
                    block_gemm_dscale<C>(Y, Z, nullptr, M, W, true, (R)-1);
                    put(tq - 1, Y);
                    block_copy(Z, Y, W * W);
                    for (int j = tq - 1; j >= 1; --j) {   // K'_{j-1} = G'_{j-1} - K'_j E_j
                        blk(M, P.E, j);
                        get(Y, j - 1);
                        __syncthreads();
                        block_gemm_dscale<C>(Y, Z, nullptr, M, W, true, (R)-1);
                        put(j - 1, Y);
                        block_copy(Z, Y, W * W);
                    }
                }
            }
            // Q = -P2 K with P2L of the level-2 separator below, P2U of the one above
            load_block(M, last ? P.P2L + (int64_t)q1 * bs : P.P2U + (int64_t)(q0 - 1) * bs, W, st.ld);
            for (int i = 0; i < n; ++i) {
                get(X, i);
                __syncthreads();
                block_gemm_dscale<C>(Y, M, nullptr, X, W, false, (R)-1);
                store_block(slot(i), Y, W, st.ld);
                __syncthreads();
            }
        }
    }
}

// Transfer composites (with separator groups): for every chunk row k of chunk p and
// transfer column c (forward to0, to1, backward to0, to1; StripDev::xc) the row vectors
//   XF[k][col][0] = GT_p(k)[c,:] GT2_{p-1},   XF[k][col][1] = GT_p(k)[c,:] GB2_{p-1},
//   XF[k][col][2] = GB_p(k)[c,:] GT2_p,       XF[k][col][3] = GB_p(k)[c,:] GB2_p
// (zero where the level-2 spike does not exist).  With them the transfer of row k
// follows from the chain solution, the group solutions of the chunk's two separators
// and the level-2 values around their groups, before those separators are final:
//   x_k[c] = y_k[c] - GT[c,:] y2_{p-1} - GB[c,:] y2_p + XF[0] x2a + XF[1] x2b + XF[2] x2a' + XF[3] x2b'.
// One CTA per (chunk, strip); two level-2 blocks staged at a time.
template <typename C>
__global__ void k_factor_xfer(Geom g, const C* __restrict__ GT, const C* __restrict__ GB,
                              const C* __restrict__ GT2, const C* __restrict__ GB2, C* __restrict__ XF) {
    const StripDev st = g.strips[blockIdx.y];
    const int p = blockIdx.x;
    const int W = st.W, SL = spld(W);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* blk = reinterpret_cast<C*>(smem_raw);   // [2][W][SL]
    const int4 m0 = g.cmeta[2 * p];
    const int r0 = m0.x, r1 = m0.y, gA = m0.z, gB = m0.w;
    const int G = g.G;
    for (int half = 0; half < 2; ++half) {   // 0: separator above (p-1), 1: separator below (p)
        const int gi = half == 0 ? gA : gB;
        const bool has[2] = {gi > 0, gi >= 0 && gi < G - 1};   // GT2, GB2 of that separator exist
        const int q = half == 0 ? p - 1 : p;
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * W * SL; e += blockDim.x) {
            const int k = e / (W * SL), o = e % (W * SL);
            blk[e] = has[k] ? (k == 0 ? GT2 : GB2)[st.red + (int64_t)q * st.bs + o] : CT<C>::zero();
        }
        __syncthreads();
        for (int k = r0; k < r1; ++k)
            for (int col = 0; col < 4; ++col) {
                const int c = st.xc[col];
                const C* v = (half == 0 ? GT : GB) + st.fac + (int64_t)k * st.bs + (int64_t)c * SL;
                for (int o = threadIdx.x; o < 2 * SL; o += blockDim.x) {
                    const int k2 = o / SL, a = o % SL;
                    C acc = CT<C>::zero();
                    if (has[k2] && a < W) {
                        const C* M = blk + k2 * W * SL + a;
                        for (int cc = 0; cc < W; ++cc) acc = cfma(v[cc], M[cc * SL], acc);
                    }
                    XF[st.xf + (((int64_t)k * 4 + col) * 4 + half * 2 + k2) * SL + a] = acc;
                }
            }
    }
}

size_t factor_smem_bytes(int Wmax, size_t esize, int nbuf) {
    return (size_t)nbuf * Wmax * Wmax * esize + (size_t)3 * Wmax * esize + (size_t)((Wmax + 3) & ~3) * 4 + 16;
}

template <typename C>
cudaError_t launch_factor(const Geom& g, int Wmax, void* const* pool, int* status, cudaStream_t s, KernelTimer* tm) {
    const size_t smem = factor_smem_bytes(Wmax, sizeof(C), 3);
    const size_t smem_sep = factor_smem_bytes(Wmax, sizeof(C), g.G > 1 ? 4 : 3);
    if (smem_sep > kFactorSmemMax) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(k_factor_chunk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_factor_sep<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sep);
    if (err != cudaSuccess) return err;
    dim3 grid(g.P, g.J);
    {
        TimedLaunch t(tm, "factor_chunk", s);
        k_factor_chunk<C><<<grid, 256, smem, s>>>(g, (C*)pool[0], (C*)pool[1], (C*)pool[2], status);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (g.P > 1) {
        SepPools<C> pl{(C*)pool[3], (C*)pool[4], (C*)pool[5], (C*)pool[6], (C*)pool[7], (C*)pool[8], (C*)pool[9],
                       g.G > 1 ? (C*)pool[11] : nullptr, g.G > 1 ? (C*)pool[12] : nullptr};
        TimedLaunch t(tm, "factor_sep", s);
        k_factor_sep<C><<<g.J, 256, smem_sep, s>>>(g, (const C*)pool[1], (const C*)pool[2], pl, status);
    }
    if (g.G > 1) {
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const size_t xs = (size_t)2 * Wmax * spld(Wmax) * sizeof(C);
        err = cudaFuncSetAttribute(k_factor_xfer<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
        if (err != cudaSuccess) return err;
        TimedLaunch t(tm, "factor_xfer", s);
        k_factor_xfer<C><<<dim3(g.P, g.J), 256, xs, s>>>(g, (const C*)pool[1], (const C*)pool[2], (const C*)pool[6],
                                                          (const C*)pool[7], (C*)pool[10]);
    }
    return cudaGetLastError();
}

template cudaError_t launch_factor<float2>(const Geom&, int, void* const*, int*, cudaStream_t, KernelTimer*);
template cudaError_t launch_factor<double2>(const Geom&, int, void* const*, int*, cudaStream_t, KernelTimer*);

}  // namespace helm
