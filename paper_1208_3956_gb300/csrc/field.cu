// FP64 grid kernels: k^2 on the padded grid, the paper-form stencil A u and the
// residual f - A u (Section 2.2), column copies (compose), the Krylov kernels of
// GMRES (batched inner products, multi-vector updates, scaling), and the misfit
// gradient accumulation / fold.
#include "common.cuh"
#include "internal.h"

namespace helm {

static inline int nblocks(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    return (int)(b > (1 << 30) ? (1 << 30) : b);
}

// ---------------------------------------------------------------- k^2
// k^2 = omega^2 / c^2 on the padded grid, c clamp-extended into the outer layer
// (Eq. helm1, k = omega / c).
__global__ void k_k2(const double* __restrict__ c, double* __restrict__ k2, int nx, int ny, int nz, int w,
                     double omega2) {
    const int Nx = nx + 2 * w, Ny = ny + 2 * w;
    const int Nz = (nz > 1 || w == 0) ? nz + (nz > 1 ? 2 * w : 0) : 1;
    const int64_t tot = (int64_t)Nx * Ny * Nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Nx);
        const int y = (int)((i / Nx) % Ny);
        const int z = (int)(i / ((int64_t)Nx * Ny));
        const int xi = min(max(x - w, 0), nx - 1);
        const int yi = min(max(y - w, 0), ny - 1);
        const int zi = (nz > 1) ? min(max(z - w, 0), nz - 1) : 0;
        const double cv = c[((int64_t)zi * ny + yi) * nx + xi];
        k2[i] = omega2 / (cv * cv);
    }
}

cudaError_t launch_k2(const double* c_int, double* k2, int dim, int nx, int ny, int nz, int w, double omega,
                      cudaStream_t s) {
    const int Nz = dim == 3 ? nz + 2 * w : 1;
    const int64_t tot = (int64_t)(nx + 2 * w) * (ny + 2 * w) * Nz;
    k_k2<<<nblocks(tot, 256), 256, 0, s>>>(c_int, k2, nx, ny, dim == 3 ? nz : 1, w, omega * omega);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- stencil
// (A u)_p = sum_axes -a(i)[a(i+1/2)(u_{i+1}-u_i) - a(i-1/2)(u_i-u_{i-1})]/h^2 - k^2 u_p
__device__ __forceinline__ double2 axis_term(double2 ai, double2 ap, double2 am, double2 u, double2 up,
                                             double2 um) {
    const double2 fwd = cmul(ap, csub(up, u));
    const double2 bwd = cmul(am, csub(u, um));
    return cneg(cmul(ai, csub(fwd, bwd)));
}

__global__ void k_stencil(Geom g, const double2* __restrict__ u, const double2* __restrict__ f,
                          double2* __restrict__ out, int B) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int64_t plane = (int64_t)Nx * Ny;
    const int64_t vol = plane * Nz;
    const int64_t tot = vol * B;
    const double2 zero = make_double2(0.0, 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i % vol;
        const int x = (int)(p % Nx);
        const int y = (int)((p / Nx) % Ny);
        const int z = (int)(p / plane);
        const double2 uc = u[i];
        double2 acc = axis_term(g.gx_int[x], g.gx_half[x + 1], g.gx_half[x], uc,
                                x + 1 < Nx ? u[i + 1] : zero, x > 0 ? u[i - 1] : zero);
        acc = cadd(acc, axis_term(g.gy_int[y], g.gy_half[y + 1], g.gy_half[y], uc,
                                  y + 1 < Ny ? u[i + Nx] : zero, y > 0 ? u[i - Nx] : zero));
        if (Nz > 1)
            acc = cadd(acc, axis_term(g.gz_int[z], g.gz_half[z + 1], g.gz_half[z], uc,
                                      z + 1 < Nz ? u[i + plane] : zero, z > 0 ? u[i - plane] : zero));
        acc = cscale(acc, g.inv_h2);
        acc = csub(acc, cscale(uc, g.k2[p]));
        out[i] = f ? csub(f[i], acc) : acc;
    }
}

cudaError_t launch_stencil(const Geom& g, const double2* u, const double2* f, double2* out, int B,
                           cudaStream_t s, KernelTimer* tm) {
    const int64_t tot = (int64_t)g.Nx * g.Ny * g.Nz * B;
    TimedLaunch t(tm, "stencil", s);
    k_stencil<<<nblocks(tot, 256), 256, 0, s>>>(g, u, f, out, B);
    return cudaGetLastError();
}

// dst(b, z, y, x) = src(b, z, y, x) for xlo <= x <= xhi
__global__ void k_copy_cols(const double2* __restrict__ src, double2* __restrict__ dst, int64_t rows, int Nx,
                            int xlo, int xhi) {
    const int w = xhi - xlo + 1;
    const int64_t tot = rows * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / w;
        const int x = xlo + (int)(i % w);
        dst[r * Nx + x] = src[r * Nx + x];
    }
}

cudaError_t launch_copy_cols(const double2* src, double2* dst, int B, int Nx, int Ny, int Nz, int xlo, int xhi,
                             cudaStream_t s, KernelTimer* tm) {
    if (xhi < xlo) return cudaSuccess;
    const int64_t rows = (int64_t)B * Ny * Nz;
    TimedLaunch t(tm, "compose_copy", s);
    k_copy_cols<<<nblocks(rows * (xhi - xlo + 1), 256), 256, 0, s>>>(src, dst, rows, Nx, xlo, xhi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Krylov
__global__ void k_multidot(const double2* __restrict__ V, int64_t vstride, const double2* __restrict__ w,
                           int nv, int B, int64_t N, double2* __restrict__ partial) {
    const int blk = blockIdx.x, i = blockIdx.y, b = blockIdx.z;
    const double2* vi = V + i * vstride + (int64_t)b * N;
    const double2* wb = w + (int64_t)b * N;
    double re = 0.0, im = 0.0;
    for (int64_t n = blk * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = vi[n], c = wb[n];
        // conj(a) * c
        re = fma(a.x, c.x, re); re = fma(a.y, c.y, re);
        im = fma(a.x, c.y, im); im = fma(-a.y, c.x, im);
    }
    __shared__ double sre[32], sim[32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sre[wid] = re; sim[wid] = im; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        re = lane < nw ? sre[lane] : 0.0;
        im = lane < nw ? sim[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) partial[((int64_t)b * nv + i) * gridDim.x + blk] = make_double2(re, im);
    }
}

// out[b*nv+i] = sum over blocks, fixed order (deterministic)
__global__ void k_reduce_partials(const double2* __restrict__ partial, int nblk, int count,
                                  double2* __restrict__ out) {
    const int id = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (id >= count) return;
    double re = 0.0, im = 0.0;
    for (int k = lane; k < nblk; k += 32) {
        const double2 v = partial[(int64_t)id * nblk + k];
        re += v.x;
        im += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) out[id] = make_double2(re, im);
}

cudaError_t launch_multidot(const double2* V, int64_t vstride, const double2* w, int nv, int B, int64_t N,
                            double2* partial, int nblk, double2* out, cudaStream_t s, KernelTimer* tm) {
    {
        TimedLaunch t(tm, "krylov_dot", s);
        k_multidot<<<dim3(nblk, nv, B), 256, 0, s>>>(V, vstride, w, nv, B, N, partial);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int count = nv * B;
    TimedLaunch t(tm, "krylov_reduce", s);
    k_reduce_partials<<<(count + 7) / 8, 256, 0, s>>>(partial, nblk, count, out);
    return cudaGetLastError();
}

__global__ void k_multi_axpy(double2* __restrict__ w, const double2* __restrict__ V, int64_t vstride,
                             const double2* __restrict__ coef, int nv, int B, int64_t N) {
    const int64_t tot = (int64_t)B * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / N);
        double2 acc = w[i];
        for (int k = 0; k < nv; ++k) acc = cfma(coef[b * nv + k], V[k * vstride + i], acc);
        w[i] = acc;
    }
}

cudaError_t launch_multi_axpy(double2* w, const double2* V, int64_t vstride, const double2* coef, int nv,
                              int B, int64_t N, cudaStream_t s, KernelTimer* tm) {
    if (nv <= 0) return cudaSuccess;
    TimedLaunch t(tm, "krylov_axpy", s);
    k_multi_axpy<<<nblocks((int64_t)B * N, 256), 256, 0, s>>>(w, V, vstride, coef, nv, B, N);
    return cudaGetLastError();
}

__global__ void k_scale(double2* __restrict__ dst, const double2* __restrict__ src,
                        const double* __restrict__ scale, int B, int64_t N) {
    const int64_t tot = (int64_t)B * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = cscale(src[i], scale[i / N]);
}

cudaError_t launch_scale(double2* dst, const double2* src, const double* scale, int B, int64_t N,
                         cudaStream_t s, KernelTimer* tm) {
    TimedLaunch t(tm, "krylov_scale", s);
    k_scale<<<nblocks((int64_t)B * N, 256), 256, 0, s>>>(dst, src, scale, B, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- misfit gradient
// gpad(p) = omega^2 Re sum_s S(p) mu_s(p) u_s(p),  S = prod_axes 1/alpha
__global__ void k_grad_accum(Geom g, const double2* __restrict__ U, const double2* __restrict__ MU, int nsrc,
                             double* __restrict__ gpad) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int64_t plane = (int64_t)Nx * Ny, vol = plane * Nz;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < vol; p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % Nx), y = (int)((p / Nx) % Ny), z = (int)(p / plane);
        double2 S = cmul(cinv(g.gx_int[x]), cinv(g.gy_int[y]));
        if (Nz > 1) S = cmul(S, cinv(g.gz_int[z]));
        double acc = 0.0;
        for (int s = 0; s < nsrc; ++s) {
            const double2 t = cmul(S, cmul(MU[(int64_t)s * vol + p], U[(int64_t)s * vol + p]));
            acc += t.x;
        }
        gpad[p] = g.omega * g.omega * acc;
    }
}

cudaError_t launch_grad_accum(const double2* U, const double2* MU, const Geom& g, int nsrc, double* gpad,
                              cudaStream_t s) {
    const int64_t vol = (int64_t)g.Nx * g.Ny * g.Nz;
    k_grad_accum<<<nblocks(vol, 256), 256, 0, s>>>(g, U, MU, nsrc, gpad);
    return cudaGetLastError();
}

// Adjoint of the clamp extension: each interior cell sums the padded cells that
// copy it.
__global__ void k_fold(const double* __restrict__ gpad, double* __restrict__ gint, int nx, int ny, int nz,
                       int w, int dim) {
    const int Nx = nx + 2 * w, Ny = ny + 2 * w;
    const int64_t tot = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        const int xa = x == 0 ? 0 : x + w, xb = x == nx - 1 ? Nx - 1 : x + w;
        const int ya = y == 0 ? 0 : y + w, yb = y == ny - 1 ? Ny - 1 : y + w;
        int za = 0, zb = 0;
        if (dim == 3) { za = z == 0 ? 0 : z + w; zb = z == nz - 1 ? nz + 2 * w - 1 : z + w; }
        double acc = 0.0;
        for (int zz = za; zz <= zb; ++zz)
            for (int yy = ya; yy <= yb; ++yy)
                for (int xx = xa; xx <= xb; ++xx) acc += gpad[((int64_t)zz * Ny + yy) * Nx + xx];
        gint[i] = acc;
    }
}

cudaError_t launch_fold(const double* gpad, double* gint, int dim, int nx, int ny, int nz, int w, cudaStream_t s) {
    const int64_t tot = (int64_t)nx * ny * (dim == 3 ? nz : 1);
    k_fold<<<nblocks(tot, 256), 256, 0, s>>>(gpad, gint, nx, ny, dim == 3 ? nz : 1, w, dim);
    return cudaGetLastError();
}

__global__ void k_gather(const double2* __restrict__ U, int64_t ustride, const int64_t* __restrict__ idx,
                         int nidx, int B, double2* __restrict__ out) {
    const int64_t tot = (int64_t)B * nidx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / nidx), r = (int)(i % nidx);
        out[i] = U[(int64_t)b * ustride + idx[r]];
    }
}

cudaError_t launch_gather(const double2* U, int64_t ustride, const int64_t* idx, int nidx, int B, double2* out,
                          cudaStream_t s) {
    k_gather<<<nblocks((int64_t)B * nidx, 256), 256, 0, s>>>(U, ustride, idx, nidx, B, out);
    return cudaGetLastError();
}

}  // namespace helm
