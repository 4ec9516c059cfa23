// One strip solve of the double sweep (Section 2.1, Eqs. solve_upward and
// solve_downward) on the partitioned block-tridiagonal factors of factor.cu.
//
//   k_sweep_chunk    one CTA per (chunk, RHS tile): builds the strip right-hand
//                    side S^(j) r (masked source plus the single-layer transfer)
//                    row by row and solves the chunk system A_p y_p = b_p by
//                    block forward elimination and back substitution.
//   k_sweep_reduced  one CTA per RHS tile: separator right-hand sides
//                    bhat_q = b_s - C_s y_q(last) - C_{s+1} y_{q+1}(first), then the
//                    separator chain z_q = Rinv_q bhat_q - E_q z_{q-1},
//                    x_q = z_q - F_q x_{q+1}.
//   k_sweep_correct  one CTA per (row, RHS tile): x_k = y_k - GT_p(k) x_{p-1} -
//                    GB_p(k) x_p, scatter to the output field (compose) and emit
//                    the transfer difference for the next strip.
#include "common.cuh"
#include "strip_ops.cuh"
#include "internal.h"

namespace helm {

static constexpr int kSweepThreads = 128;

struct SweepArgs {
    Geom g;
    StripDev st;
    SweepStep sp;
    int Wmax, B, Bt;
};

// FP64 right-hand side entry of S^(j) r for strip-local column c, row k, RHS b.
__device__ __forceinline__ double2 strip_rhs(const SweepArgs& A, int k, int c, int b) {
    const StripDev& st = A.st;
    const int gc = st.lo - st.lpml + c;
    double2 v = make_double2(0.0, 0.0);
    const int64_t row = ((int64_t)b * A.g.Ny + k);
    if (gc >= A.sp.mlo && gc <= A.sp.mhi) v = A.sp.src[row * A.g.Nx + gc];
    if (A.sp.tin && (gc == A.sp.t0 || gc == A.sp.t0 + 1)) v = cadd(v, cscale(A.sp.tin[row], A.sp.tcoef));
    return cmul(v, cmul(strip_sx(A.g, st, c), glob_sy(A.g, k)));
}

template <typename C>
__device__ __forceinline__ C* yrow(void* ybuf, const SweepArgs& A, int b, int k) {
    return reinterpret_cast<C*>(ybuf) + ((int64_t)b * A.g.Ny + k) * A.Wmax;
}

template <typename C>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_chunk(SweepArgs A, const C* __restrict__ Sinv,
                                                               void* ybuf) {
    const int p = blockIdx.x;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int r0 = A.g.r0[p], r1 = A.g.r1[p];
    const C* S = Sinv + A.st.fac;
    const int64_t bs = A.st.bs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* t = reinterpret_cast<C*>(smem_raw);   // W*Bt
    C* zp = t + W * A.Bt;                      // W*Bt
    const int nout = W * nb;

    // forward elimination: z_k = Sinv_k (b_k - C_k z_{k-1})
    for (int k = r0; k < r1; ++k) {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            C r = CT<C>::from(strip_rhs(A, k, c, b0 + bb));
            if (k > r0) r = csub(r, cmul(CT<C>::from(strip_coupling(A.g, A.st, k, c)), zp[o]));
            t[o] = r;
        }
        __syncthreads();
        const C* Sk = S + (int64_t)k * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            const C* tv = t + bb * W;
            C acc = CT<C>::zero();
            for (int a = 0; a < W; ++a) acc = cfma(Sk[a * W + c], tv[a], acc);
            zp[o] = acc;
            yrow<C>(ybuf, A, b0 + bb, k)[c] = acc;
        }
        __syncthreads();
    }
    // back substitution: x_k = z_k - Sinv_k C_{k+1} x_{k+1}; zp holds x_{r1-1}
    for (int k = r1 - 2; k >= r0; --k) {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W;
            t[o] = cmul(CT<C>::from(strip_coupling(A.g, A.st, k + 1, c)), zp[o]);
        }
        __syncthreads();
        const C* Sk = S + (int64_t)k * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            const C* tv = t + bb * W;
            C* yk = yrow<C>(ybuf, A, b0 + bb, k);
            C acc = yk[c];
            C s = CT<C>::zero();
            for (int a = 0; a < W; ++a) s = cfma(Sk[a * W + c], tv[a], s);
            acc = csub(acc, s);
            zp[o] = acc;
            yk[c] = acc;
        }
        __syncthreads();
    }
}

template <typename C>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_reduced(SweepArgs A, const C* __restrict__ Rinv,
                                                                 const C* __restrict__ E,
                                                                 const C* __restrict__ F, void* ybuf) {
    const int b0 = blockIdx.x * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int nout = W * nb;
    const int64_t bs = A.st.bs;
    const C* Rs = Rinv + A.st.red;
    const C* Es = E + A.st.red;
    const C* Fs = F + A.st.red;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* t = reinterpret_cast<C*>(smem_raw);   // W*Bt
    C* zp = t + W * A.Bt;
    const int Q = A.g.P - 1;

    // a_q = Rinv_q bhat_q, parked in the separator rows of ybuf
    for (int q = 0; q < Q; ++q) {
        const int s = A.g.r1[q];
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            C r = CT<C>::from(strip_rhs(A, s, c, b0 + bb));
            const C ylast = yrow<C>(ybuf, A, b0 + bb, s - 1)[c];
            const C yfirst = yrow<C>(ybuf, A, b0 + bb, s + 1)[c];
            r = csub(r, cmul(CT<C>::from(strip_coupling(A.g, A.st, s, c)), ylast));
            r = csub(r, cmul(CT<C>::from(strip_coupling(A.g, A.st, s + 1, c)), yfirst));
            t[o] = r;
        }
        __syncthreads();
        const C* Rq = Rs + (int64_t)q * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            const C* tv = t + bb * W;
            C acc = CT<C>::zero();
            for (int a = 0; a < W; ++a) acc = cfma(Rq[a * W + c], tv[a], acc);
            yrow<C>(ybuf, A, b0 + bb, s)[c] = acc;
        }
        __syncthreads();
    }
    // forward chain z_q = a_q - E_q z_{q-1}
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int c = o % W, bb = o / W;
        zp[o] = yrow<C>(ybuf, A, b0 + bb, A.g.r1[0])[c];
    }
    __syncthreads();
    for (int q = 1; q < Q; ++q) {
        const int s = A.g.r1[q];
        const C* Eq = Es + (int64_t)q * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            const C* zv = zp + bb * W;
            C acc = CT<C>::zero();
            for (int a = 0; a < W; ++a) acc = cfma(Eq[a * W + c], zv[a], acc);
            t[o] = csub(yrow<C>(ybuf, A, b0 + bb, s)[c], acc);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            zp[o] = t[o];
            yrow<C>(ybuf, A, b0 + bb, s)[c] = t[o];
        }
        __syncthreads();
    }
    // backward chain x_q = z_q - F_q x_{q+1}; zp holds x_{Q-1}
    for (int q = Q - 2; q >= 0; --q) {
        const int s = A.g.r1[q];
        const C* Fq = Fs + (int64_t)q * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            const C* xv = zp + bb * W;
            C acc = CT<C>::zero();
            for (int a = 0; a < W; ++a) acc = cfma(Fq[a * W + c], xv[a], acc);
            t[o] = csub(yrow<C>(ybuf, A, b0 + bb, s)[c], acc);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            zp[o] = t[o];
            yrow<C>(ybuf, A, b0 + bb, s)[c] = t[o];
        }
        __syncthreads();
    }
}

template <typename C>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_correct(SweepArgs A, const C* __restrict__ GT,
                                                                 const C* __restrict__ GB, void* ybuf) {
    const int k = blockIdx.x;
    const int b0 = blockIdx.y * A.Bt;
    const int nb = imin(A.Bt, A.B - b0);
    const int W = A.st.W;
    const int nout = W * nb;
    const int64_t bs = A.st.bs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xa = reinterpret_cast<C*>(smem_raw);  // separator above (W*Bt)
    C* xb = xa + W * A.Bt;                     // separator below
    C* xs = xb + W * A.Bt;                     // the row's solution
    const int pm = A.g.rowmap[k];
    const bool has_above = pm > 0;
    const bool has_below = pm >= 0 && pm < A.g.P - 1;
    if (pm >= 0) {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            if (has_above) xa[o] = yrow<C>(ybuf, A, b0 + bb, A.g.r1[pm - 1])[c];
            if (has_below) xb[o] = yrow<C>(ybuf, A, b0 + bb, A.g.r1[pm])[c];
        }
        __syncthreads();
        const C* GTk = GT + A.st.fac + (int64_t)k * bs;
        const C* GBk = GB + A.st.fac + (int64_t)k * bs;
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            C acc = yrow<C>(ybuf, A, b0 + bb, k)[c];
            C s = CT<C>::zero();
            if (has_above) {
                const C* xv = xa + bb * W;
                for (int a = 0; a < W; ++a) s = cfma(GTk[a * W + c], xv[a], s);
            }
            if (has_below) {
                const C* xv = xb + bb * W;
                for (int a = 0; a < W; ++a) s = cfma(GBk[a * W + c], xv[a], s);
            }
            xs[o] = csub(acc, s);
        }
    } else {
        for (int o = threadIdx.x; o < nout; o += blockDim.x) {
            const int c = o % W, bb = o / W;
            xs[o] = yrow<C>(ybuf, A, b0 + bb, k)[c];
        }
    }
    __syncthreads();
    // scatter (compose) and the outgoing transfer difference
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int c = o % W, bb = o / W;
        const int gc = A.st.lo - A.st.lpml + c;
        const int64_t row = (int64_t)(b0 + bb) * A.g.Ny + k;
        if (gc >= A.sp.olo && gc <= A.sp.ohi) {
            double2 v = to_d2(xs[o]);
            if (A.sp.base) v = cadd(v, A.sp.base[row * A.g.Nx + gc]);
            A.sp.dst[row * A.g.Nx + gc] = v;
        }
        if (A.sp.tout && c == A.sp.to1)
            A.sp.tout[row] = csub(to_d2(xs[o]), to_d2(xs[bb * W + A.sp.to0]));
    }
}

template <typename C>
cudaError_t launch_strip_solve(const Geom& g, int j, const StripDev& st, const SweepStep& step,
                               const SweepWork& wk, const void* Sinv, const void* GT, const void* GB,
                               const void* Rinv, const void* E, const void* F, cudaStream_t s,
                               KernelTimer* tm) {
    SweepArgs A;
    A.g = g;
    A.st = st;
    A.sp = step;
    A.Wmax = wk.Wmax;
    A.B = wk.B;
    A.Bt = imin(wk.B, 8);
    const int ntile = (wk.B + A.Bt - 1) / A.Bt;
    const size_t smem2 = (size_t)2 * st.W * A.Bt * sizeof(C);
    const size_t smem3 = (size_t)3 * st.W * A.Bt * sizeof(C);
    {
        TimedLaunch t(tm, "sweep_chunk", s);
        k_sweep_chunk<C><<<dim3(g.P, ntile), kSweepThreads, smem2, s>>>(A, (const C*)Sinv, wk.ybuf);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (g.P > 1) {
        TimedLaunch t(tm, "sweep_reduced", s);
        k_sweep_reduced<C><<<ntile, kSweepThreads, smem2, s>>>(A, (const C*)Rinv, (const C*)E, (const C*)F,
                                                               wk.ybuf);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    {
        TimedLaunch t(tm, "sweep_correct", s);
        k_sweep_correct<C><<<dim3(g.Ny, ntile), kSweepThreads, smem3, s>>>(A, (const C*)GT, (const C*)GB,
                                                                          wk.ybuf);
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
