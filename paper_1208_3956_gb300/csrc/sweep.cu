// One strip solve of the double sweep (Section 2.1, Eqs. solve_upward and
// solve_downward) on the partitioned block-tridiagonal factors of factor.cu.
//
// k_sweep_chunk (grid: chunks x RHS tiles)
//   * builds the strip right-hand side S^(j) r for every row of its chunk
//     (masked source plus the single-layer-potential transfer on two columns);
//   * streams the chunk's Sinv_k blocks global -> shared memory with TMA bulk
//     copies (cp.async.bulk + mbarrier ring; the whole chunk stays resident when
//     it fits, so the back substitution reads no HBM);
//   * runs the chain z_k = Sinv_k (b_k - C_k z_{k-1}), x_k = z_k - Sinv_k C_{k+1} x_{k+1}
//     with the W x W products split over the warps (lanes own rows);
//   * adds its two parts of the separator right-hand sides, Rinv_q times
//     (b_s - C_s y_q(last)) and -Rinv_q C_{s+1} y_{q+1}(first);
//   * the last CTA of a tile to finish (atomic arrival counter, no waiting)
//     solves the separator system z_q = a_q - E_q z_{q-1}, x_q = z_q - F_q x_{q+1}.
// k_sweep_correct (grid: rows x RHS tiles)
//   x_k = y_k - GT_p(k) x_{p-1} - GB_p(k) x_p on the output columns only, scatter
//   to the output field (compose) and emit the transfer difference.
//
// Every mbarrier wait is bounded; on time-out the kernel records
// HELM_ETIMEOUT in the status word, drains its copies (bounded) and returns.
#include "common.cuh"
#include "internal.h"

namespace helm {

static constexpr int kNW = 4;                 // warps per CTA
static constexpr int kThreads = 32 * kNW;
static constexpr int kMaxRing = 32;
static constexpr uint32_t kWaitLimit = 1u << 22;

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

// ------------------------------------------------------------------ args
struct SweepArgs {
    Geom g;
    StripDev st;
    SweepStep sp;
    int Wmax, B, Bt;
    int ring;                // slots of the block ring
    int zrows;               // rows of the z buffer (max chunk rows, separators)
    uint32_t slot_bytes;     // bytes of one staged W x W block
    const void* Sinv;
    const void* Rinv;
    const void* E;
    const void* F;
    void* ybuf;              // [B][Ny][Wmax] chunk solutions, then separator values
    void* parts;             // [B][P-1][2][Wmax] separator right-hand-side parts
    int* counters;           // [ntile] arrival counters, left at zero
    int* status;
};

template <typename C>
__device__ __forceinline__ const C* ctab(const Geom& g) { return reinterpret_cast<const C*>(g.ct); }

template <typename C>
__device__ __forceinline__ C coupling(const SweepArgs& A, int k, int c) {
    return cmul(ctab<C>(A.g)[A.st.ctab + c], ctab<C>(A.g)[A.g.ct_cy + k]);
}

// S^(j) r at strip-local column c, row k, RHS b (working precision)
template <typename C>
__device__ __forceinline__ C rhs_entry(const SweepArgs& A, int k, int c, int b) {
    const int gc = A.st.lo - A.st.lpml + c;
    double2 v = make_double2(0.0, 0.0);
    const int64_t row = (int64_t)b * A.g.Ny + k;
    if (gc >= A.sp.mlo && gc <= A.sp.mhi) v = A.sp.src[row * A.g.Nx + gc];
    if (A.sp.tin && (gc == A.sp.t0 || gc == A.sp.t0 + 1)) {
        const double2 t = A.sp.tin[row];
        v.x = fma(A.sp.tcoef, t.x, v.x);
        v.y = fma(A.sp.tcoef, t.y, v.y);
    }
    return cmul(CT<C>::from(v), cmul(ctab<C>(A.g)[A.st.ctab + c], ctab<C>(A.g)[A.g.ct_sy + k]));
}

template <typename C>
__device__ __forceinline__ C* yrow(const SweepArgs& A, int b, int k) {
    return reinterpret_cast<C*>(A.ybuf) + ((int64_t)b * A.g.Ny + k) * A.Wmax;
}

// Shared-memory carve-up (bytes), identical on host and device.
struct SweepSmem {
    uint32_t slots, zb, tv, red, mbar, flags, total;
};
__host__ __device__ inline SweepSmem sweep_smem(int ring, uint32_t slot_bytes, int zrows, int Bt, int W,
                                                int esz) {
    SweepSmem s;
    uint32_t o = 0;
    s.slots = o; o += ring * slot_bytes;
    s.zb = o; o += ((uint32_t)zrows * Bt * W * esz + 15u) & ~15u;
    s.tv = o; o += (uint32_t)Bt * 64 * esz;
    s.red = o; o += (uint32_t)kNW * Bt * 64 * esz;
    s.mbar = o; o += kMaxRing * 8;
    s.flags = o; o += 16;
    s.total = o;
    return s;
}

// Block ring: load number G goes to slot G % ring with parity (G / ring) & 1.
template <typename C>
struct Ring {
    unsigned char* slots;
    uint64_t* mbar;
    int ring;
    uint32_t slot_bytes;
    __device__ C* slot(int G) const { return reinterpret_cast<C*>(slots + (size_t)(G % ring) * slot_bytes); }
    __device__ void issue(int G, const C* src) const {   // one thread
        uint64_t* m = &mbar[G % ring];
        fence_proxy_async();
        mbar_expect_tx(m, slot_bytes);
        bulk_g2s(slots + (size_t)(G % ring) * slot_bytes, src, slot_bytes, m);
    }
    __device__ bool wait(int G) const { return mbar_wait(&mbar[G % ring], (uint32_t)((G / ring) & 1)); }
};

// partial products red[w][b][r] = sum_{a in warp w's range} S(r,a) t[b][a]
template <typename C>
__device__ __forceinline__ void warp_partial(const C* __restrict__ S, const C* __restrict__ tv, C* red, int W,
                                             int nb, int Bt) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int per = (W + kNW - 1) / kNW;
    const int a0 = w * per, a1 = imin(W, a0 + per);
    const bool r0ok = l < W, r1ok = l + 32 < W;
    for (int b = 0; b < nb; ++b) {
        const C* tb = tv + b * 64;
        C e0 = CT<C>::zero(), o0 = CT<C>::zero(), e1 = CT<C>::zero(), o1 = CT<C>::zero();
        int a = a0;
        for (; a + 1 < a1; a += 2) {
            const C t0 = tb[a], t1 = tb[a + 1];
            if (r0ok) { e0 = cfma(S[a * W + l], t0, e0); o0 = cfma(S[(a + 1) * W + l], t1, o0); }
            if (r1ok) { e1 = cfma(S[a * W + l + 32], t0, e1); o1 = cfma(S[(a + 1) * W + l + 32], t1, o1); }
        }
        if (a < a1) {
            const C t0 = tb[a];
            if (r0ok) e0 = cfma(S[a * W + l], t0, e0);
            if (r1ok) e1 = cfma(S[a * W + l + 32], t0, e1);
        }
        C* rb = red + (w * Bt + b) * 64;
        rb[l] = cadd(e0, o0);
        rb[l + 32] = cadd(e1, o1);
    }
}

template <typename C>
__device__ __forceinline__ C red_sum(const C* red, int b, int c, int Bt) {
    C s = red[b * 64 + c];
#pragma unroll
    for (int w = 1; w < kNW; ++w) s = cadd(s, red[(w * Bt + b) * 64 + c]);
    return s;
}

__device__ __forceinline__ bool block_any(bool v) { return __syncthreads_or(v ? 1 : 0) != 0; }

// ------------------------------------------------------------------ chunk + separators
template <typename C>
__global__ void __launch_bounds__(kThreads) k_sweep_chunk(SweepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = A.st.W;
    const int esz = (int)sizeof(C);
    const SweepSmem L = sweep_smem(A.ring, A.slot_bytes, A.zrows, A.Bt, W, esz);
    Ring<C> R{smem + L.slots, reinterpret_cast<uint64_t*>(smem + L.mbar), A.ring, A.slot_bytes};
    C* zb = reinterpret_cast<C*>(smem + L.zb);       // [zrows][Bt][W]
    C* tv = reinterpret_cast<C*>(smem + L.tv);       // [Bt][64]
    C* red = reinterpret_cast<C*>(smem + L.red);     // [NW][Bt][64]
    int* flags = reinterpret_cast<int*>(smem + L.flags);
    const int p = blockIdx.x, tile = blockIdx.y;
    const int b0 = tile * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int r0 = A.g.r0[p], r1 = A.g.r1[p], m = r1 - r0;
    const int P = A.g.P, Q = P - 1;
    const int tid = threadIdx.x;
    const int64_t bs = A.st.bs;
    const C* Sinv = reinterpret_cast<const C*>(A.Sinv) + A.st.fac;
    const C* Rinv = reinterpret_cast<const C*>(A.Rinv) + A.st.red;
    const bool resident = A.ring >= m + 2;
    // load schedule of this CTA: forward blocks r0..r1-1, (ring mode) backward
    // blocks r1-2..r0, then Rinv_p (separator below) and Rinv_{p-1} (above).
    const int nfwd = m, nbwd = resident ? 0 : m - 1;
    const bool has_below = p < P - 1, has_above = p > 0;
    const int nload = nfwd + nbwd + (has_below ? 1 : 0) + (has_above ? 1 : 0);
    auto block_of = [&](int G) -> const C* {
        if (G < nfwd) return Sinv + (int64_t)(r0 + G) * bs;
        G -= nfwd;
        if (G < nbwd) return Sinv + (int64_t)(r1 - 2 - G) * bs;
        G -= nbwd;
        if (has_below && G == 0) return Rinv + (int64_t)p * bs;
        return Rinv + (int64_t)(p - 1) * bs;
    };
    if (tid == 0) {
        for (int i = 0; i < A.ring; ++i) mbar_init(&R.mbar[i], 1);
        fence_mbar_init();
        for (int G = 0; G < imin(A.ring, nload); ++G) R.issue(G, block_of(G));
    }
    // right-hand sides of every chunk row (independent of the chain)
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        zb[(r * A.Bt + b) * W + c] = rhs_entry<C>(A, r0 + r, c, b0 + b);
    }
    __syncthreads();
    for (int o = tid; o < nb * W; o += blockDim.x) {
        const int c = o % W, b = o / W;
        tv[b * 64 + c] = zb[b * W + c];
    }
    __syncthreads();
    int G = 0;              // next load to consume
    int issued = imin(A.ring, nload);   // loads issued so far (thread 0's count)
    int pending_lo = 0;     // first load not yet consumed (for the drain on time-out)
    bool bad = false;
    auto consume = [&](int Gc) -> const C* {
        pending_lo = Gc;
        if (!R.wait(Gc)) bad = true;
        else pending_lo = Gc + 1;
        return R.slot(Gc);
    };
    auto issue = [&](int Gi, const C* src) {
        R.issue(Gi, src);
        issued = Gi + 1;
    };
    // bounded wait gave up: record HELM_ETIMEOUT, wait (bounded) for the copies
    // issued but not consumed, then the caller returns
    auto drain = [&]() {
        if (tid == 0) {
            atomicExch(A.status, 7);
            for (int Gd = pending_lo; Gd < issued; ++Gd) R.wait(Gd);
        }
        __syncthreads();
    };
    // ---- forward elimination
    for (int s = 0; s < m; ++s) {
        const int k = r0 + s;
        const C* S = consume(G);
        if (block_any(bad)) { drain(); return; }
        warp_partial(S, tv, red, W, nb, A.Bt);
        __syncthreads();
        if (tid == 0 && !resident && G + A.ring < nload) issue(G + A.ring, block_of(G + A.ring));
        ++G;
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            const C z = red_sum(red, b, c, A.Bt);
            zb[(s * A.Bt + b) * W + c] = z;
            if (s + 1 < m) tv[b * 64 + c] = csub(zb[((s + 1) * A.Bt + b) * W + c], cmul(coupling<C>(A, k + 1, c), z));
            else tv[b * 64 + c] = cmul(coupling<C>(A, k, c), z);   // C_{k+1} x_{k+1} for the back substitution
        }
        __syncthreads();
    }
    // ---- back substitution
    for (int s = m - 2; s >= 0; --s) {
        const int k = r0 + s;
        const C* S;
        if (resident) S = R.slot(s);
        else S = consume(G);
        if (block_any(bad)) { drain(); return; }
        warp_partial(S, tv, red, W, nb, A.Bt);
        __syncthreads();
        if (!resident) {
            if (tid == 0 && G + A.ring < nload) issue(G + A.ring, block_of(G + A.ring));
            ++G;
        }
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            const C x = csub(zb[(s * A.Bt + b) * W + c], red_sum(red, b, c, A.Bt));
            zb[(s * A.Bt + b) * W + c] = x;
            tv[b * 64 + c] = cmul(coupling<C>(A, k, c), x);
        }
        __syncthreads();
    }
    // ---- chunk solution to global memory
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        yrow<C>(A, b0 + b, r0 + r)[c] = zb[(r * A.Bt + b) * W + c];
    }
    // ---- separator right-hand-side parts: A_p = Rinv_p (b_s - C_s y(last)), s = r1
    //      and B_{p-1} = -Rinv_{p-1} C_{s'+1} y(first), s' = r0 - 1
    if (Q > 0) {
        C* parts = reinterpret_cast<C*>(A.parts);
        for (int part = 0; part < 2; ++part) {
            const bool active = part == 0 ? has_below : has_above;
            if (!active) continue;
            for (int o = tid; o < nb * W; o += blockDim.x) {
                const int c = o % W, b = o / W;
                C t;
                if (part == 0) {
                    const int s = r1;
                    t = csub(rhs_entry<C>(A, s, c, b0 + b), cmul(coupling<C>(A, s, c), zb[((m - 1) * A.Bt + b) * W + c]));
                } else {
                    const int s = r0 - 1;
                    t = cneg(cmul(coupling<C>(A, s + 1, c), zb[b * W + c]));
                }
                tv[b * 64 + c] = t;
            }
            __syncthreads();
            const C* S = consume(G);
            if (block_any(bad)) { drain(); return; }
            ++G;
            warp_partial(S, tv, red, W, nb, A.Bt);
            __syncthreads();
            const int q = part == 0 ? p : p - 1;
            for (int o = tid; o < nb * W; o += blockDim.x) {
                const int c = o % W, b = o / W;
                parts[((((int64_t)(b0 + b) * Q + q) * 2 + part) * A.Wmax) + c] = red_sum(red, b, c, A.Bt);
            }
            __syncthreads();
        }
    }
    if (Q == 0) return;
    // ---- arrival: the last CTA of this tile solves the separator system
    __threadfence();
    __syncthreads();
    if (tid == 0) flags[0] = (atomicAdd(&A.counters[tile], 1) == P - 1) ? 1 : 0;
    __syncthreads();
    if (!flags[0]) return;
    __threadfence();
    {
        const C* parts = reinterpret_cast<const C*>(A.parts);
        const C* E = reinterpret_cast<const C*>(A.E) + A.st.red;
        const C* F = reinterpret_cast<const C*>(A.F) + A.st.red;
        // loads continue the same ring sequence: E_1..E_{Q-1}, F_{Q-2}..F_0
        const int G0 = nload;
        const int nred = 2 * (Q - 1);
        auto rblock = [&](int Gr) -> const C* {
            const int i = Gr - G0;
            if (i < Q - 1) return E + (int64_t)(1 + i) * bs;
            return F + (int64_t)(Q - 2 - (i - (Q - 1))) * bs;
        };
        if (tid == 0)
            for (int Gr = G0; Gr < G0 + imin(A.ring, nred); ++Gr) issue(Gr, rblock(Gr));
        // a_q = A_q + B_q into zb[q]
        for (int o = tid; o < Q * nb * W; o += blockDim.x) {
            const int c = o % W, b = (o / W) % nb, q = o / (W * nb);
            const int64_t base = (((int64_t)(b0 + b) * Q + q) * 2) * A.Wmax + c;
            zb[(q * A.Bt + b) * W + c] = cadd(__ldcg(parts + base), __ldcg(parts + base + A.Wmax));
        }
        __syncthreads();
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            tv[b * 64 + c] = zb[b * W + c];
        }
        __syncthreads();
        int Gr = G0;
        // forward: z_q = a_q - E_q z_{q-1}
        for (int q = 1; q < Q; ++q) {
            const C* S = consume(Gr);
            if (block_any(bad)) { drain(); return; }
            warp_partial(S, tv, red, W, nb, A.Bt);
            __syncthreads();
            if (tid == 0 && Gr + A.ring < G0 + nred) issue(Gr + A.ring, rblock(Gr + A.ring));
            ++Gr;
            for (int o = tid; o < nb * W; o += blockDim.x) {
                const int c = o % W, b = o / W;
                const C z = csub(zb[(q * A.Bt + b) * W + c], red_sum(red, b, c, A.Bt));
                zb[(q * A.Bt + b) * W + c] = z;
                tv[b * 64 + c] = z;
            }
            __syncthreads();
        }
        // backward: x_q = z_q - F_q x_{q+1}
        for (int q = Q - 2; q >= 0; --q) {
            const C* S = consume(Gr);
            if (block_any(bad)) { drain(); return; }
            warp_partial(S, tv, red, W, nb, A.Bt);
            __syncthreads();
            if (tid == 0 && Gr + A.ring < G0 + nred) issue(Gr + A.ring, rblock(Gr + A.ring));
            ++Gr;
            for (int o = tid; o < nb * W; o += blockDim.x) {
                const int c = o % W, b = o / W;
                const C x = csub(zb[(q * A.Bt + b) * W + c], red_sum(red, b, c, A.Bt));
                zb[(q * A.Bt + b) * W + c] = x;
                tv[b * 64 + c] = x;
            }
            __syncthreads();
        }
        for (int o = tid; o < Q * nb * W; o += blockDim.x) {
            const int c = o % W, b = (o / W) % nb, q = o / (W * nb);
            yrow<C>(A, b0 + b, A.g.r1[q])[c] = zb[(q * A.Bt + b) * W + c];
        }
        if (tid == 0) A.counters[tile] = 0;
    }
}

// ------------------------------------------------------------------ correction
template <typename C>
__global__ void __launch_bounds__(kThreads) k_sweep_correct(SweepArgs A, const C* __restrict__ GT,
                                                            const C* __restrict__ GB) {
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int64_t bs = A.st.bs;
    __shared__ __align__(16) C xa[4 * 64];
    __shared__ __align__(16) C xb[4 * 64];
    __shared__ __align__(16) C xs[4 * 64];
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int pm = A.g.rowmap[k];
    // output columns (strip-local) plus the transfer columns
    const int off = A.st.lo - A.st.lpml;
    const int olo = imax(A.sp.olo - off, 0), ohi = imin(A.sp.ohi - off, W - 1);
    const int nout = imax(ohi - olo + 1, 0);
    int extra[2];
    int nextra = 0;
    if (A.sp.tout) {
        if (A.sp.to0 < olo || A.sp.to0 > ohi) extra[nextra++] = A.sp.to0;
        if (A.sp.to1 < olo || A.sp.to1 > ohi) extra[nextra++] = A.sp.to1;
    }
    const int ncol = nout + nextra;
    auto col = [&](int i) { return i < nout ? olo + i : extra[i - nout]; };
    if (pm < 0) {
        for (int o = tid; o < nb * ncol; o += blockDim.x) {
            const int c = col(o % ncol), b = o / ncol;
            xs[b * 64 + c] = yrow<C>(A, b0 + b, k)[c];
        }
    } else {
        const bool above = pm > 0, below = pm < A.g.P - 1;
        for (int o = tid; o < nb * W; o += blockDim.x) {
            const int c = o % W, b = o / W;
            if (above) xa[b * 64 + c] = yrow<C>(A, b0 + b, A.g.r1[pm - 1])[c];
            if (below) xb[b * 64 + c] = yrow<C>(A, b0 + b, A.g.r1[pm])[c];
        }
        __syncthreads();
        const C* GTk = GT + A.st.fac + (int64_t)k * bs;
        const C* GBk = GB + A.st.fac + (int64_t)k * bs;
        for (int i = w; i < ncol; i += kNW) {
            const int c = col(i);
            for (int b = 0; b < nb; ++b) {
                C s = CT<C>::zero();
                for (int a = l; a < W; a += 32) {
                    if (above) s = cfma(GTk[(int64_t)c * W + a], xa[b * 64 + a], s);
                    if (below) s = cfma(GBk[(int64_t)c * W + a], xb[b * 64 + a], s);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                }
                if (l == 0) xs[b * 64 + c] = csub(yrow<C>(A, b0 + b, k)[c], s);
            }
        }
    }
    __syncthreads();
    for (int o = tid; o < nb * nout; o += blockDim.x) {
        const int c = olo + o % nout, b = o / nout;
        const int gc = off + c;
        const int64_t row = (int64_t)(b0 + b) * A.g.Ny + k;
        double2 v = to_d2(xs[b * 64 + c]);
        if (A.sp.base) v = cadd(v, A.sp.base[row * A.g.Nx + gc]);
        A.sp.dst[row * A.g.Nx + gc] = v;
    }
    if (A.sp.tout)
        for (int b = tid; b < nb; b += blockDim.x)
            A.sp.tout[(int64_t)(b0 + b) * A.g.Ny + k] =
                csub(to_d2(xs[b * 64 + A.sp.to1]), to_d2(xs[b * 64 + A.sp.to0]));
}

// ------------------------------------------------------------------ host
template <typename C>
static SweepArgs make_args(const Geom& g, const StripDev& st, const SweepStep& step, const SweepWork& wk,
                           const void* Sinv, const void* Rinv, const void* E, const void* F, int Bt, int ring) {
    SweepArgs A;
    A.g = g;
    A.st = st;
    A.sp = step;
    A.Wmax = wk.Wmax;
    A.B = wk.B;
    A.Bt = Bt;
    A.ring = ring;
    A.zrows = wk.zrows;
    A.slot_bytes = (uint32_t)(st.bs * sizeof(C));
    A.Sinv = Sinv;
    A.Rinv = Rinv;
    A.E = E;
    A.F = F;
    A.ybuf = wk.ybuf;
    A.parts = wk.parts;
    A.counters = wk.counters;
    A.status = wk.status;
    return A;
}

// Largest ring (and RHS tile) that fits the shared-memory budget.
template <typename C>
static bool plan(const StripDev& st, int zrows, int B, int& Bt, int& ring, size_t& smem) {
    const size_t budget = 220 * 1024;
    const uint32_t slot = (uint32_t)(st.bs * sizeof(C));
    for (Bt = imin(B, 4); Bt >= 1; --Bt) {
        for (ring = kMaxRing; ring >= 2; --ring) {
            smem = sweep_smem(ring, slot, zrows, Bt, st.W, (int)sizeof(C)).total;
            if (smem <= budget) return true;
        }
    }
    return false;
}

template <typename C>
cudaError_t launch_strip_solve(const Geom& g, int j, const StripDev& st, const SweepStep& step,
                               const SweepWork& wk, const void* Sinv, const void* GT, const void* GB,
                               const void* Rinv, const void* E, const void* F, cudaStream_t s,
                               KernelTimer* tm) {
    int Bt, ring;
    size_t smem;
    if (!plan<C>(st, wk.zrows, wk.B, Bt, ring, smem)) return cudaErrorInvalidConfiguration;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_chunk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    SweepArgs A = make_args<C>(g, st, step, wk, Sinv, Rinv, E, F, Bt, ring);
    const int ntile = (wk.B + Bt - 1) / Bt;
    {
        TimedLaunch t(tm, "sweep_chunk", s);
        k_sweep_chunk<C><<<dim3(g.P, ntile), kThreads, smem, s>>>(A);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    {
        TimedLaunch t(tm, "sweep_correct", s);
        k_sweep_correct<C><<<dim3(g.Ny, ntile), kThreads, 0, s>>>(A, (const C*)GT, (const C*)GB);
    }
    return cudaGetLastError();
}

template cudaError_t launch_strip_solve<float2>(const Geom&, int, const StripDev&, const SweepStep&,
                                                const SweepWork&, const void*, const void*, const void*,
                                                const void*, const void*, const void*, cudaStream_t,
                                                KernelTimer*);
template cudaError_t launch_strip_solve<double2>(const Geom&, int, const StripDev&, const SweepStep&,
                                                 const SweepWork&, const void*, const void*, const void*,
                                                 const void*, const void*, const void*, cudaStream_t,
                                                 KernelTimer*);

}  // namespace helm
