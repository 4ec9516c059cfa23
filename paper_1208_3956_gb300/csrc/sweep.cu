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
    uint32_t slots, zb, tv, tv2, cx, cy, mbar, flags, total;
};
__host__ __device__ inline SweepSmem sweep_smem(int ring, uint32_t slot_bytes, int zrows, int Bt, int W,
                                                int esz) {
    SweepSmem s;
    uint32_t o = 0;
    s.slots = o; o += ring * slot_bytes;
    s.zb = o; o += ((uint32_t)zrows * Bt * W * esz + 15u) & ~15u;
    s.tv = o; o += (uint32_t)Bt * 64 * esz;
    s.tv2 = o; o += (uint32_t)Bt * 64 * esz;
    s.cx = o; o += 64u * esz;
    s.cy = o; o += ((uint32_t)(zrows + 2) * esz + 15u) & ~15u;
    s.mbar = o; o += kMaxRing * 8;
    s.flags = o; o += 16;
    s.total = o;
    return s;
}

// ------------------------------------------------------------------ chunk + separators
// Matrix-vector layout of one chain step: the CTA has ceil(W/8) warps; lane l of
// warp w owns row r = 8w + l/4 and the columns a = l%4 + 4j, j < NJ, of the
// column-major W x W block in shared memory.  Offsets are precomputed once and
// clamped into the block (a clamped column meets a zero entry of the vector, a
// clamped row is computed but never stored), and two xor shuffles complete the
// row sums.
template <typename C, int NJ>
__global__ void __launch_bounds__(256) k_sweep_chunk(SweepArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = A.st.W;
    const int esz = (int)sizeof(C);
    const SweepSmem L = sweep_smem(A.ring, A.slot_bytes, A.zrows, A.Bt, W, esz);
    unsigned char* slots = smem + L.slots;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);
    C* zb = reinterpret_cast<C*>(smem + L.zb);       // [zrows][Bt][W]
    C* tin = reinterpret_cast<C*>(smem + L.tv);      // [Bt][64] vector entering the step
    C* tout = reinterpret_cast<C*>(smem + L.tv2);    // [Bt][64] vector entering the next step
    C* csx = reinterpret_cast<C*>(smem + L.cx);      // s_x(c)
    C* ccy = reinterpret_cast<C*>(smem + L.cy);      // -alpha_y(k-1/2)/h^2, k = r0..r1
    volatile int* flags = reinterpret_cast<int*>(smem + L.flags);
    const int p = blockIdx.x, tile = blockIdx.y;
    const int b0 = tile * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int r0 = A.g.r0[p], r1 = A.g.r1[p], m = r1 - r0;
    const int P = A.g.P, Q = P - 1;
    const int tid = threadIdx.x;
    const int64_t bs = A.st.bs;
    const int Bt = A.Bt;
    const int ring = A.ring;
    const uint32_t sb = A.slot_bytes;
    const C* Sinv = reinterpret_cast<const C*>(A.Sinv) + A.st.fac;
    const C* Rinv = reinterpret_cast<const C*>(A.Rinv) + A.st.red;
    const bool resident = ring >= m + 2;
    // load schedule: forward blocks r0..r1-1, (streaming mode) backward blocks
    // r1-2..r0, then Rinv_p (separator below) and Rinv_{p-1} (separator above).
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
    // ---- ring state: loads are numbered G; load G lives in slot G % ring and
    // completes phase (G / ring) & 1 of that slot's barrier.
    int issued = 0;                 // thread 0: loads issued
    int consumed = 0;               // loads consumed (waited for)
    int cslot = 0;                  // slot of load `consumed`
    uint32_t cpar = 0;              // its phase parity
    int last_slot = 0;              // slot of the last consumed load
    auto issue_into = [&](int slot, const C* src) {   // thread 0 only
        uint64_t* mb = &mbar[slot];
        fence_proxy_async();
        mbar_expect_tx(mb, sb);
        bulk_g2s(slots + (size_t)slot * sb, src, sb, mb);
        ++issued;
    };
    auto consume = [&]() -> const C* {
        const C* S = reinterpret_cast<const C*>(slots + (size_t)cslot * sb);
        if (!mbar_wait(&mbar[cslot], cpar)) flags[1] = 1;
        last_slot = cslot;
        ++consumed;
        if (++cslot == ring) { cslot = 0; cpar ^= 1u; }
        return S;
    };
    // a bounded wait gave up (flags[1], read after a barrier, so uniform):
    // record HELM_ETIMEOUT, wait (bounded) for the copies still in flight
    auto drain = [&]() {
        if (tid == 0) {
            atomicExch(A.status, 7);
            for (int Gd = consumed - 1; Gd < issued; ++Gd)
                if (Gd >= 0) mbar_wait(&mbar[Gd % ring], (uint32_t)((Gd / ring) & 1));
        }
        __syncthreads();
    };
    if (tid == 0) {
        flags[1] = 0;
        for (int i = 0; i < ring; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
        for (int G = 0; G < imin(ring, nload); ++G) issue_into(G, block_of(G));
    }
    const C* ct = ctab<C>(A.g);
    for (int o = tid; o < 2 * Bt * 64; o += blockDim.x) tin[o] = CT<C>::zero();   // tin, tout are adjacent
    for (int c = tid; c < W; c += blockDim.x) csx[c] = ct[A.st.ctab + c];
    for (int k = r0 + tid; k <= r1; k += blockDim.x) ccy[k - r0] = ct[A.g.ct_cy + k];
    __syncthreads();
    // right-hand sides of every chunk row (independent of the chain)
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        const C v = rhs_entry<C>(A, r0 + r, c, b0 + b);
        zb[(r * Bt + b) * W + c] = v;
        if (r == 0) tin[b * 64 + c] = v;
    }
    // per-lane geometry of the products
    const int w = tid >> 5, l = tid & 31;
    const int row = w * 8 + (l >> 2);
    const int g = l & 3;
    const bool own = g == 0 && row < W;
    const int rc = imin(row, W - 1);
    int soff[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) soff[j] = imin(g + 4 * j, W - 1) * W + rc;
    const C csx_r = csx[rc];
    __syncthreads();
    // v_b = sum_a S(row, a) t_b(a) for b < nb; calls fn(b, v) on the owning lane
    auto step = [&](const C* S, const C* t, auto fn) {
        C sr[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) sr[j] = S[soff[j]];
        for (int b = 0; b < nb; ++b) {
            const C* tb = t + b * 64 + g;
            C a0 = CT<C>::zero(), a1 = CT<C>::zero();
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {
                a0 = cfma(sr[j], tb[4 * j], a0);
                if (j + 1 < NJ) a1 = cfma(sr[j + 1], tb[4 * j + 4], a1);
            }
            C v = cadd(a0, a1);
            v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
            v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
            v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
            if (own) fn(b, v);
        }
    };
    auto cy = [&](int k) -> C { return ccy[k - r0]; };
    int G = 0;   // next load number to consume (also drives the refills)
    // ---- forward elimination z_k = Sinv_k (b_k - C_k z_{k-1})
    for (int s = 0; s < m; ++s) {
        const int k = r0 + s;
        const C* S = consume();
        const C ck = cmul(csx_r, cy(s + 1 < m ? k + 1 : k));
        step(S, tin, [&](int b, C v) {
            zb[(s * Bt + b) * W + row] = v;
            tout[b * 64 + row] = (s + 1 < m) ? csub(zb[((s + 1) * Bt + b) * W + row], cmul(ck, v))
                                             : cmul(ck, v);   // C_{k+1} x_{k+1} for the back substitution
        });
        __syncthreads();
        if (flags[1]) { drain(); return; }
        if (tid == 0 && !resident && G + ring < nload) issue_into(last_slot, block_of(G + ring));
        ++G;
        C* t = tin; tin = tout; tout = t;
    }
    // ---- back substitution x_k = z_k - Sinv_k C_{k+1} x_{k+1}
    for (int s = m - 2; s >= 0; --s) {
        const int k = r0 + s;
        const C* S = resident ? reinterpret_cast<const C*>(slots + (size_t)s * sb) : consume();
        const C ck = cmul(csx_r, cy(k));
        step(S, tin, [&](int b, C v) {
            const C x = csub(zb[(s * Bt + b) * W + row], v);
            zb[(s * Bt + b) * W + row] = x;
            tout[b * 64 + row] = cmul(ck, x);
        });
        __syncthreads();
        if (flags[1]) { drain(); return; }
        if (!resident) {
            if (tid == 0 && G + ring < nload) issue_into(last_slot, block_of(G + ring));
            ++G;
        }
        C* t = tin; tin = tout; tout = t;
    }
    // ---- chunk solution to global memory
    for (int o = tid; o < m * nb * W; o += blockDim.x) {
        const int c = o % W, b = (o / W) % nb, r = o / (W * nb);
        yrow<C>(A, b0 + b, r0 + r)[c] = zb[(r * Bt + b) * W + c];
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
                if (part == 0)
                    t = csub(rhs_entry<C>(A, r1, c, b0 + b),
                             cmul(cmul(csx[c], cy(r1)), zb[((m - 1) * Bt + b) * W + c]));
                else
                    t = cneg(cmul(cmul(csx[c], cy(r0)), zb[b * W + c]));
                tin[b * 64 + c] = t;
            }
            __syncthreads();
            const C* S = consume();
            const int q = part == 0 ? p : p - 1;
            step(S, tin, [&](int b, C v) {
                parts[((((int64_t)(b0 + b) * Q + q) * 2 + part) * A.Wmax) + row] = v;
            });
            __syncthreads();
            if (flags[1]) { drain(); return; }
            if (tid == 0 && !resident && G + ring < nload) issue_into(last_slot, block_of(G + ring));
            ++G;
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
        const int nred = 2 * (Q - 1);
        auto rblock = [&](int i) -> const C* {
            if (i < Q - 1) return E + (int64_t)(1 + i) * bs;
            return F + (int64_t)(Q - 2 - (i - (Q - 1))) * bs;
        };
        // every earlier load has been consumed: continue from slot `cslot`
        if (tid == 0) {
            int sl = cslot;
            for (int i = 0; i < imin(ring, nred); ++i) {
                issue_into(sl, rblock(i));
                if (++sl == ring) sl = 0;
            }
        }
        // a_q = A_q + B_q
        for (int o = tid; o < Q * nb * W; o += blockDim.x) {
            const int c = o % W, b = (o / W) % nb, q = o / (W * nb);
            const int64_t base = (((int64_t)(b0 + b) * Q + q) * 2) * A.Wmax + c;
            const C v = cadd(__ldcg(parts + base), __ldcg(parts + base + A.Wmax));
            zb[(q * Bt + b) * W + c] = v;
            if (q == 0) tin[b * 64 + c] = v;
        }
        __syncthreads();
        int i = 0;   // separator-load counter
        // forward: z_q = a_q - E_q z_{q-1}
        for (int q = 1; q < Q; ++q) {
            const C* S = consume();
            step(S, tin, [&](int b, C v) {
                const C z = csub(zb[(q * Bt + b) * W + row], v);
                zb[(q * Bt + b) * W + row] = z;
                tout[b * 64 + row] = z;
            });
            __syncthreads();
            if (flags[1]) { drain(); return; }
            if (tid == 0 && i + ring < nred) issue_into(last_slot, rblock(i + ring));
            ++i;
            C* t = tin; tin = tout; tout = t;
        }
        // backward: x_q = z_q - F_q x_{q+1}
        for (int q = Q - 2; q >= 0; --q) {
            const C* S = consume();
            step(S, tin, [&](int b, C v) {
                const C x = csub(zb[(q * Bt + b) * W + row], v);
                zb[(q * Bt + b) * W + row] = x;
                tout[b * 64 + row] = x;
            });
            __syncthreads();
            if (flags[1]) { drain(); return; }
            if (tid == 0 && i + ring < nred) issue_into(last_slot, rblock(i + ring));
            ++i;
            C* t = tin; tin = tout; tout = t;
        }
        for (int o = tid; o < Q * nb * W; o += blockDim.x) {
            const int c = o % W, b = (o / W) % nb, q = o / (W * nb);
            yrow<C>(A, b0 + b, A.g.r1[q])[c] = zb[(q * Bt + b) * W + c];
        }
        if (tid == 0) A.counters[tile] = 0;
    }
}

// ------------------------------------------------------------------ correction
// One CTA per (row, RHS tile); 8 lanes per output column read the spike rows
// GT_p(k)[c, :], GB_p(k)[c, :] (row-major, coalesced) against the separator
// values, a three-level butterfly finishes the dot products, and the owning
// lane scatters x (plus the base field) to the output.
template <typename C>
__global__ void __launch_bounds__(256) k_sweep_correct(SweepArgs A, const C* __restrict__ GT,
                                                       const C* __restrict__ GB) {
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int64_t bs = A.st.bs;
    __shared__ C xt[8];   // the two transfer columns, per RHS (Bt <= 4)
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int pm = A.g.rowmap[k];
    const int off = A.st.lo - A.st.lpml;
    const int olo = imax(A.sp.olo - off, 0), ohi = imin(A.sp.ohi - off, W - 1);
    const int nout = imax(ohi - olo + 1, 0);
    const bool tr = A.sp.tout != nullptr;
    const bool x0 = tr && (A.sp.to0 < olo || A.sp.to0 > ohi);
    const bool x1 = tr && (A.sp.to1 < olo || A.sp.to1 > ohi);
    const int ncol = nout + (x0 ? 1 : 0) + (x1 ? 1 : 0);
    const bool above = pm > 0, below = pm >= 0 && pm < A.g.P - 1;
    const int g = l & 7;
    const int64_t rowoff = (int64_t)k * bs;
    for (int base = w * 4; base < ncol; base += (blockDim.x >> 5) * 4) {   // warp-uniform trip count
        // column i of this 8-lane group; groups past ncol idle but join the shuffles
        const int i = base + (l >> 3);
        const bool live = i < ncol;
        int c = 0;
        if (live) {
            if (i < nout) c = olo + i;
            else if (i == nout && x0) c = A.sp.to0;
            else c = A.sp.to1;
        }
        for (int b = 0; b < nb; ++b) {
            C s = CT<C>::zero();
            if (live && pm >= 0) {
                const C* xa = yrow<C>(A, b0 + b, above ? A.g.r1[pm - 1] : 0);
                const C* xb = yrow<C>(A, b0 + b, below ? A.g.r1[pm] : 0);
                for (int a = g; a < W; a += 8) {
                    if (above) s = cfma(GT[A.st.fac + rowoff + (int64_t)c * W + a], xa[a], s);
                    if (below) s = cfma(GB[A.st.fac + rowoff + (int64_t)c * W + a], xb[a], s);
                }
            }
            s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
            s.x += __shfl_xor_sync(0xffffffffu, s.x, 2);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, 2);
            s.x += __shfl_xor_sync(0xffffffffu, s.x, 4);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, 4);
            if (live && g == 0) {
                const C x = csub(yrow<C>(A, b0 + b, k)[c], s);
                const int64_t rowi = (int64_t)(b0 + b) * A.g.Ny + k;
                if (c >= olo && c <= ohi) {
                    double2 v = to_d2(x);
                    if (A.sp.base) v = cadd(v, A.sp.base[rowi * A.g.Nx + off + c]);
                    A.sp.dst[rowi * A.g.Nx + off + c] = v;
                }
                if (tr && c == A.sp.to0) xt[b * 2] = x;
                if (tr && c == A.sp.to1) xt[b * 2 + 1] = x;
            }
        }
    }
    if (!tr) return;
    __syncthreads();
    for (int b = tid; b < nb; b += blockDim.x)
        A.sp.tout[(int64_t)(b0 + b) * A.g.Ny + k] = csub(to_d2(xt[b * 2 + 1]), to_d2(xt[b * 2]));
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
        for (auto fn : {k_sweep_chunk<C, 8>, k_sweep_chunk<C, 12>, k_sweep_chunk<C, 16>}) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
            if (e != cudaSuccess) return e;
        }
        attr_set = true;
    }
    SweepArgs A = make_args<C>(g, st, step, wk, Sinv, Rinv, E, F, Bt, ring);
    const int ntile = (wk.B + Bt - 1) / Bt;
    {
        TimedLaunch t(tm, "sweep_chunk", s);
        const dim3 grid(g.P, ntile);
        const int nthr = 32 * ((st.W + 7) / 8);
        if (st.W <= 32) k_sweep_chunk<C, 8><<<grid, nthr, smem, s>>>(A);
        else if (st.W <= 48) k_sweep_chunk<C, 12><<<grid, nthr, smem, s>>>(A);
        else k_sweep_chunk<C, 16><<<grid, nthr, smem, s>>>(A);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    {
        TimedLaunch t(tm, "sweep_correct", s);
        // one warp per output column (the strip's output range plus the transfer columns)
        const int ncol = (step.ohi - step.olo + 1) + 2;
        const int nthr = 32 * imin(8, imax(1, (ncol + 3) / 4));
        k_sweep_correct<C><<<dim3(g.Ny, ntile), nthr, 0, s>>>(A, (const C*)GT, (const C*)GB);
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
