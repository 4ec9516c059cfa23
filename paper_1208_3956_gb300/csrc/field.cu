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
// (A u)_p = sum_axes [cm(i) u_{i-1} + c0(i) u_i + cp(i) u_{i+1}] - k^2 u_p with the
// per-axis entries of Geom::stc_* (Section 2.2, paper form; u = 0 beyond the grid).
//
// On GB300 the FP64 pipe, not HBM, bounds this kernel, so it is organised to issue
// few FP64 instructions per point: a thread owns one x column of a tile of kRows
// rows and marches along y with u(y-1), u(y), u(y+1) in registers (each value is
// loaded once), takes its x neighbours from the adjacent lanes by shuffles, and
// outside every PML (all entries exactly {-1, 2, -1}/h^2) evaluates
//   (2 dim / h^2 - k^2) u - (sum of the 2 dim neighbours) / h^2
// (13 FP64 instructions per point in 2-D, against 25 for the general complex form).
constexpr int kStencilRows = 16;
constexpr int kStencilThreads = 128;

__device__ __forceinline__ double2 shfl_c(double2 v, int delta, bool up) {
    double2 r;
    r.x = up ? __shfl_up_sync(0xffffffffu, v.x, delta) : __shfl_down_sync(0xffffffffu, v.x, delta);
    r.y = up ? __shfl_up_sync(0xffffffffu, v.y, delta) : __shfl_down_sync(0xffffffffu, v.y, delta);
    return r;
}

template <bool Z>
__global__ void __launch_bounds__(kStencilThreads) k_stencil(Geom g, const double2* __restrict__ u,
                                                             const double2* __restrict__ f,
                                                             double2* __restrict__ out) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int x = blockIdx.x * kStencilThreads + threadIdx.x;
    const bool on = x < Nx;
    const int xc = on ? x : Nx - 1;
    const int lane = threadIdx.x & 31;
    const int y0 = blockIdx.y * kStencilRows, y1 = min(y0 + kStencilRows, Ny);
    const int bz = blockIdx.z;
    const int z = bz % Nz;
    const int64_t plane = (int64_t)Nx * Ny;
    const int64_t pbase = (int64_t)bz * plane;          // field offset of plane (b, z)
    const double* k2 = g.k2 + (int64_t)z * plane;
    const double2 zero = make_double2(0.0, 0.0);
    const double ih2 = g.inv_h2;
    const double2 cxm = g.stc_x[3 * xc], cx0 = g.stc_x[3 * xc + 1], cxp = g.stc_x[3 * xc + 2];
    const bool xplain = x >= g.fx0 && x < g.fx1;
    double2 czm = zero, cz0 = zero, czp = zero;
    bool zplain = true;
    if (Z) {
        czm = g.stc_z[3 * z];
        cz0 = g.stc_z[3 * z + 1];
        czp = g.stc_z[3 * z + 2];
        zplain = z >= g.fz0 && z < g.fz1;
    }
    const double dplain = (Z ? 6.0 : 4.0) * ih2;
    const double2* up = u + pbase + xc;
    double2 um = (y0 > 0 && on) ? up[(int64_t)(y0 - 1) * Nx] : zero;
    double2 uc = on ? up[(int64_t)y0 * Nx] : zero;
    for (int y = y0; y < y1; ++y) {
        const int64_t row = (int64_t)y * Nx;
        const double2 un = (y + 1 < Ny && on) ? up[row + Nx] : zero;
        // x neighbours: adjacent lanes, the warp's edge lanes from memory
        double2 uxm = shfl_c(uc, 1, true), uxp = shfl_c(uc, 1, false);
        if (lane == 0) uxm = (on && x > 0) ? up[row - 1] : zero;
        if (lane == 31 || x == Nx - 1) uxp = (on && x + 1 < Nx) ? up[row + 1] : zero;
        double2 uzm = zero, uzp = zero;
        if (Z) {
            uzm = (on && z > 0) ? up[row - plane] : zero;
            uzp = (on && z + 1 < Nz) ? up[row + plane] : zero;
        }
        const double kk = on ? k2[row + xc] : 0.0;
        double2 acc;
        if (xplain && y >= g.fy0 && y < g.fy1 && zplain) {
            double2 sn = cadd(cadd(uxm, uxp), cadd(um, un));
            if (Z) sn = cadd(sn, cadd(uzm, uzp));
            const double d = dplain - kk;
            acc.x = fma(d, uc.x, -ih2 * sn.x);
            acc.y = fma(d, uc.y, -ih2 * sn.y);
        } else {
            const double2 cym = g.stc_y[3 * y], cy0 = g.stc_y[3 * y + 1], cyp = g.stc_y[3 * y + 2];
            double2 dg = cadd(cx0, cy0);
            if (Z) dg = cadd(dg, cz0);
            dg.x -= kk;
            acc = cmul(dg, uc);
            acc = cfma(cxm, uxm, acc);
            acc = cfma(cxp, uxp, acc);
            acc = cfma(cym, um, acc);
            acc = cfma(cyp, un, acc);
            if (Z) {
                acc = cfma(czm, uzm, acc);
                acc = cfma(czp, uzp, acc);
            }
        }
        if (on) {
            const int64_t i = pbase + row + x;
            out[i] = f ? csub(f[i], acc) : acc;
        }
        um = uc;
        uc = un;
    }
}

cudaError_t launch_stencil(const Geom& g, const double2* u, const double2* f, double2* out, int B,
                           cudaStream_t s, KernelTimer* tm) {
    const dim3 grid((g.Nx + kStencilThreads - 1) / kStencilThreads, (g.Ny + kStencilRows - 1) / kStencilRows,
                    (unsigned)((int64_t)B * g.Nz));
    if ((int64_t)B * g.Nz > 65535) return cudaErrorInvalidConfiguration;
    TimedLaunch t(tm, "stencil", s);
    if (g.Nz > 1)
        k_stencil<true><<<grid, kStencilThreads, 0, s>>>(g, u, f, out);
    else
        k_stencil<false><<<grid, kStencilThreads, 0, s>>>(g, u, f, out);
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
// gpad(p) += omega^2 Re sum_s S(p) mu_s(p) u_s(p),  S = prod_axes 1/alpha
__global__ void k_grad_accum(Geom g, const double2* __restrict__ U, const double2* __restrict__ MU, int nsrc,
                             double* __restrict__ gpad) {   // adds to gpad
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
        gpad[p] += g.omega * g.omega * acc;
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

// dst[b * stride + idx[b][i]] = val[b][i] for i < n: point values of B fields (the host
// merges repeated indices of a field, so every store of one index writes one value)
__global__ void k_scatter(double2* __restrict__ dst, int64_t stride, const int64_t* __restrict__ idx,
                          const double2* __restrict__ val, int n, int B) {
    const int64_t tot = (int64_t)B * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
        dst[(i / n) * stride + idx[i]] = val[i];
}

cudaError_t launch_scatter(double2* dst, int64_t stride, const int64_t* idx, const double2* val, int n, int B,
                           cudaStream_t s) {
    if (n <= 0 || B <= 0) return cudaSuccess;
    k_scatter<<<nblocks((int64_t)B * n, 256), 256, 0, s>>>(dst, stride, idx, val, n, B);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- interface lines
// The reduced space of Section 2.3 holds a field on L grid columns (the 2(J-1) lines
// beta_j+1, beta_j+2): red[r * L + i] is column cols[i] of grid row r, r running over
// the B * N_z * N_y rows of B fields.
__global__ void k_gather_cols(const double2* __restrict__ full, double2* __restrict__ red,
                              const int* __restrict__ cols, int L, int64_t rows, int Nx) {
    const int64_t tot = rows * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
        red[i] = full[(i / L) * Nx + cols[i % L]];
}

__global__ void k_scatter_cols(const double2* __restrict__ red, double2* __restrict__ full,
                               const int* __restrict__ cols, int L, int64_t rows, int Nx) {
    const int64_t tot = rows * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
        full[(i / L) * Nx + cols[i % L]] = red[i];
}

// out[r * L + i] = f - (A u) at column cols[i] of row r (paper form, the entries of
// Geom::stc_*), with f the full field f_full at that point or f_red[r * L + i]; when
// both are null, out = A u there.
__global__ void k_stencil_cols(Geom g, const double2* __restrict__ u, const double2* __restrict__ f_full,
                               const double2* __restrict__ f_red, double2* __restrict__ out,
                               const int* __restrict__ cols, int L, int B) {
    const int Nx = g.Nx, Ny = g.Ny, Nz = g.Nz;
    const int64_t plane = (int64_t)Nx * Ny;
    const int64_t rows = (int64_t)B * Nz * Ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / L;
        const int x = cols[i % L];
        const int y = (int)(r % Ny);
        const int z = (int)((r / Ny) % Nz);
        const int64_t p = r * Nx + x;
        const double2 uc = u[p];
        double2 dg = cadd(g.stc_x[3 * x + 1], g.stc_y[3 * y + 1]);
        if (Nz > 1) dg = cadd(dg, g.stc_z[3 * z + 1]);
        dg.x -= g.k2[(int64_t)z * plane + (int64_t)y * Nx + x];
        double2 acc = cmul(dg, uc);
        if (x > 0) acc = cfma(g.stc_x[3 * x], u[p - 1], acc);
        if (x + 1 < Nx) acc = cfma(g.stc_x[3 * x + 2], u[p + 1], acc);
        if (y > 0) acc = cfma(g.stc_y[3 * y], u[p - Nx], acc);
        if (y + 1 < Ny) acc = cfma(g.stc_y[3 * y + 2], u[p + Nx], acc);
        if (Nz > 1) {
            if (z > 0) acc = cfma(g.stc_z[3 * z], u[p - plane], acc);
            if (z + 1 < Nz) acc = cfma(g.stc_z[3 * z + 2], u[p + plane], acc);
        }
        if (f_full || f_red) acc = csub(f_full ? f_full[p] : f_red[i], acc);
        out[i] = acc;
    }
}

// dst += src over n entries
__global__ void k_add(double2* __restrict__ dst, const double2* __restrict__ src, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = cadd(dst[i], src[i]);
}

cudaError_t launch_gather_cols(const double2* full, double2* red, const int* cols, int L, int64_t rows, int Nx,
                               cudaStream_t s, KernelTimer* tm) {
    if (L <= 0 || rows <= 0) return cudaSuccess;
    TimedLaunch t(tm, "iface_gather", s);
    k_gather_cols<<<nblocks(rows * L, 256), 256, 0, s>>>(full, red, cols, L, rows, Nx);
    return cudaGetLastError();
}

cudaError_t launch_scatter_cols(const double2* red, double2* full, const int* cols, int L, int64_t rows, int Nx,
                                cudaStream_t s, KernelTimer* tm) {
    if (L <= 0 || rows <= 0) return cudaSuccess;
    TimedLaunch t(tm, "iface_scatter", s);
    k_scatter_cols<<<nblocks(rows * L, 256), 256, 0, s>>>(red, full, cols, L, rows, Nx);
    return cudaGetLastError();
}

cudaError_t launch_stencil_cols(const Geom& g, const double2* u, const double2* f_full, const double2* f_red,
                                double2* out, const int* cols, int L, int B, cudaStream_t s, KernelTimer* tm) {
    const int64_t rows = (int64_t)B * g.Nz * g.Ny;
    if (L <= 0 || rows <= 0) return cudaSuccess;
    TimedLaunch t(tm, "iface_stencil", s);
    k_stencil_cols<<<nblocks(rows * L, 256), 256, 0, s>>>(g, u, f_full, f_red, out, cols, L, B);
    return cudaGetLastError();
}

cudaError_t launch_add(double2* dst, const double2* src, int64_t n, cudaStream_t s, KernelTimer* tm) {
    TimedLaunch t(tm, "field_add", s);
    k_add<<<nblocks(n, 256), 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

// Loads this file's module onto the current device.
cudaError_t preload_field_kernels() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, k_copy_cols);
}

}  // namespace helm
