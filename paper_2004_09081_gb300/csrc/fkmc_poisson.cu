// fkmc_poisson.cu -- electrostatic potential of the vacancy charges for the
// mu-scale model of arXiv:2004.09081 (Sec. "Oxygen diffusion in mu-scale
// BaTiO3 model": the potential comes from a Poisson equation).  The source is
// read as the vacancies' own charge q e, split in halves between the two B
// nodes (cell corners) of each vacancy's O-site bond, against a uniform
// background; the grid is periodic with spacing a:
//
//     6 phi(n) - sum_{6 neighbours} phi(n') = Q(n) / (eps0 eps_r a)        [V]
//
// solved by a geometric multigrid V-cycle (vertex-centred coarsening by 2
// while every dimension is even; red-black Gauss-Seidel where all dimensions
// of a level are even, damped Jacobi otherwise and on the coarsest level;
// full-weighting restriction, trilinear prolongation).  Every reduction is
// deterministic (block partials summed in a fixed order), so a solve is
// reproducible bit for bit.  The potential then enters the hop rates through
// the site-energy field: u(s) = rint(q phi(s) 1e4), phi(s) the mean of the
// two nodes of site s.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fkmc_device.cuh"
#include "fkmc_kernels.h"

namespace fkmc {

namespace {

constexpr int PT = 256;

__device__ __forceinline__ int64_t nidx(int x, int y, int z, int nx, int ny) { return ((int64_t)z * ny + y) * nx + x; }

__device__ __forceinline__ int wrap_(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// integer half-charge counts: +1 at each end node of every vacancy's bond
__global__ void k_mg_deposit(RepDesc D, const VacRec* recs, const int32_t* counts, int cap, int32_t* cnt)
{
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nfrag * cap;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = D.frag_base + k / cap;
        const int slot = (int)(k % cap);
        if (slot >= counts[g]) continue;
        int t, x, y, z;
        split_key(recs[g * cap + slot].key, t, x, y, z);
        atomicAdd(cnt + nidx(x, y, z, D.L[0], D.L[1]), 1);
        const int x2 = wrap_(x + (t == 0), D.L[0]), y2 = wrap_(y + (t == 1), D.L[1]), z2 = wrap_(z + (t == 2), D.L[2]);
        atomicAdd(cnt + nidx(x2, y2, z2, D.L[0], D.L[1]), 1);
    }
}

// f = (q/2 cnt - background) * scale, background = q N_V / cells
__global__ void k_mg_rhs(const int32_t* cnt, int64_t n, double half_q, double background, double scale, double* f)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = __dmul_rn(__dadd_rn(__dmul_rn(half_q, (double)cnt[i]), -background), scale);
}

// red-black Gauss-Seidel half-sweep (all dimensions even: the colouring is
// consistent across the periodic seams)
__global__ void k_mg_rb(double* phi, const double* f, int nx, int ny, int nz, int colour)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        if (((x + y + z) & 1) != colour) continue;
        double s = phi[nidx(wrap_(x - 1, nx), y, z, nx, ny)];
        s = __dadd_rn(s, phi[nidx(wrap_(x + 1, nx), y, z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, wrap_(y - 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, wrap_(y + 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, y, wrap_(z - 1, nz), nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, y, wrap_(z + 1, nz), nx, ny)]);
        phi[i] = __ddiv_rn(__dadd_rn(f[i], s), 6.0);
    }
}

// damped Jacobi sweep, out = (1-w) in + w (f + sum nb) / 6
__global__ void k_mg_jacobi(const double* in, double* out, const double* f, int nx, int ny, int nz, double w)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        double s = in[nidx(wrap_(x - 1, nx), y, z, nx, ny)];
        s = __dadd_rn(s, in[nidx(wrap_(x + 1, nx), y, z, nx, ny)]);
        s = __dadd_rn(s, in[nidx(x, wrap_(y - 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, in[nidx(x, wrap_(y + 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, in[nidx(x, y, wrap_(z - 1, nz), nx, ny)]);
        s = __dadd_rn(s, in[nidx(x, y, wrap_(z + 1, nz), nx, ny)]);
        const double gs = __ddiv_rn(__dadd_rn(f[i], s), 6.0);
        out[i] = __dadd_rn(__dmul_rn(1.0 - w, in[i]), __dmul_rn(w, gs));
    }
}

// r = f - A phi
__global__ void k_mg_residual(const double* phi, const double* f, double* r, int nx, int ny, int nz)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        double s = phi[nidx(wrap_(x - 1, nx), y, z, nx, ny)];
        s = __dadd_rn(s, phi[nidx(wrap_(x + 1, nx), y, z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, wrap_(y - 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, wrap_(y + 1, ny), z, nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, y, wrap_(z - 1, nz), nx, ny)]);
        s = __dadd_rn(s, phi[nidx(x, y, wrap_(z + 1, nz), nx, ny)]);
        r[i] = __dadd_rn(f[i], -__dadd_rn(__dmul_rn(6.0, phi[i]), -s));
    }
}

// coarse f = 4 x full weighting of the fine residual (weights (1,2,1)^3 / 64)
__global__ void k_mg_restrict(const double* r, double* fc, int nx, int ny, int nz)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t n = (int64_t)cx * cy * cz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % cx), Y = (int)((i / cx) % cy), Z = (int)(i / ((int64_t)cx * cy));
        double s = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const double w = (double)((2 - (dx != 0)) * (2 - (dy != 0)) * (2 - (dz != 0)));
                    s = __dadd_rn(s, __dmul_rn(w, r[nidx(wrap_(2 * X + dx, nx), wrap_(2 * Y + dy, ny),
                                                         wrap_(2 * Z + dz, nz), nx, ny)]));
                }
        fc[i] = __dmul_rn(s, 4.0 / 64.0);
    }
}

// phi_fine += trilinear interpolation of the coarse correction
__global__ void k_mg_prolong(const double* ec, double* phi, int nx, int ny, int nz)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        const int X = x >> 1, Y = y >> 1, Z = z >> 1, ox = x & 1, oy = y & 1, oz = z & 1;
        double s = 0.0;
        for (int dz = 0; dz <= oz; ++dz)
            for (int dy = 0; dy <= oy; ++dy)
                for (int dx = 0; dx <= ox; ++dx)
                    s = __dadd_rn(s, ec[nidx(wrap_(X + dx, cx), wrap_(Y + dy, cy), wrap_(Z + dz, cz), cx, cy)]);
        phi[i] = __dadd_rn(phi[i], __dmul_rn(s, 1.0 / (double)(1 << (ox + oy + oz))));
    }
}

// deterministic sum: per-block partials (fixed grid), then one thread in order
__global__ void k_mg_partial(const double* v, int64_t n, double* part, int absmax)
{
    __shared__ double sh[PT];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * PT + threadIdx.x; i < n; i += (int64_t)gridDim.x * PT)
        s = absmax ? fmax(s, fabs(v[i])) : __dadd_rn(s, v[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = PT / 2; w; w >>= 1) {
        if (threadIdx.x < w)
            sh[threadIdx.x] = absmax ? fmax(sh[threadIdx.x], sh[threadIdx.x + w])
                                     : __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mg_final(const double* part, int nb, double* out, int absmax)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s = absmax ? fmax(s, part[b]) : __dadd_rn(s, part[b]);
    *out = s;
}

// v -= sum / n (sum from k_mg_final)
__global__ void k_mg_sub_mean(double* v, int64_t n, const double* sum)
{
    const double m = __ddiv_rn(*sum, (double)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = __dadd_rn(v[i], -m);
}

// u(s) = rint(q phi(s) 1e4) per O site of replica D, phi(s) the mean of the two
// nodes of its bond; the energy field moves by the change; |u| max recorded
__global__ void k_elec_update(RepDesc D, const double* phi, double q, int32_t* u, int32_t* field, unsigned* umax)
{
    const int nx = D.L[0], ny = D.L[1], nz = D.L[2];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < D.nsite; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)((s / ((int64_t)nx * ny)) % nz);
        const int t = (int)(s / ((int64_t)nx * ny * nz));
        const double p2 = phi[nidx(wrap_(x + (t == 0), nx), wrap_(y + (t == 1), ny), wrap_(z + (t == 2), nz), nx, ny)];
        const double ps = __dmul_rn(0.5, __dadd_rn(phi[nidx(x, y, z, nx, ny)], p2));
        const int32_t un = (int32_t)__double2ll_rn(__dmul_rn(__dmul_rn(q, ps), 1e4));
        const int64_t gs = D.site_off + s;
        if (field) field[gs] += un - u[gs];
        u[gs] = un;
        atomicMax(umax, (unsigned)(un < 0 ? -un : un));
    }
}

// field += u (after the field was rebuilt from the vacancies and dopants)
__global__ void k_elec_add(int32_t* field, const int32_t* u, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        field[i] += u[i];
}

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + PT - 1) / PT, 8192)); }

}  // namespace

MgPlan mg_plan(int nx, int ny, int nz)
{
    MgPlan p{};
    int dims[3] = {nx, ny, nz};
    int64_t off = 0;
    for (p.levels = 0; p.levels < MG_MAX_LEVELS; ++p.levels) {
        for (int d = 0; d < 3; ++d) p.dim[p.levels][d] = dims[d];
        p.off[p.levels] = off;
        off += (int64_t)dims[0] * dims[1] * dims[2];
        const bool even = dims[0] % 2 == 0 && dims[1] % 2 == 0 && dims[2] % 2 == 0;
        if (!even || dims[0] < 4 || dims[1] < 4 || dims[2] < 4) {
            ++p.levels;
            break;
        }
        for (int d = 0; d < 3; ++d) dims[d] /= 2;
    }
    p.total = off;
    return p;
}

static bool level_even(const MgPlan& p, int l)
{
    return p.dim[l][0] % 2 == 0 && p.dim[l][1] % 2 == 0 && p.dim[l][2] % 2 == 0;
}

static void smooth(const MgPlan& p, int l, const MgBuffers& b, int sweeps, cudaStream_t st)
{
    const int nx = p.dim[l][0], ny = p.dim[l][1], nz = p.dim[l][2];
    const int64_t n = (int64_t)nx * ny * nz;
    double* phi = b.phi + p.off[l];
    const double* f = b.f + p.off[l];
    for (int k = 0; k < sweeps; ++k) {
        if (level_even(p, l)) {
            k_mg_rb<<<grid_for(n), PT, 0, st>>>(phi, f, nx, ny, nz, 0);
            k_mg_rb<<<grid_for(n), PT, 0, st>>>(phi, f, nx, ny, nz, 1);
        } else {  // two Jacobi half-steps through the scratch level buffer
            double* tmp = b.r + p.off[l];
            k_mg_jacobi<<<grid_for(n), PT, 0, st>>>(phi, tmp, f, nx, ny, nz, 6.0 / 7.0);
            k_mg_jacobi<<<grid_for(n), PT, 0, st>>>(tmp, phi, f, nx, ny, nz, 6.0 / 7.0);
        }
    }
}

static void sub_mean(double* v, int64_t n, const MgBuffers& b, cudaStream_t st)
{
    k_mg_partial<<<MG_PARTIALS, PT, 0, st>>>(v, n, b.part, 0);
    k_mg_final<<<1, 32, 0, st>>>(b.part, MG_PARTIALS, b.scalar, 0);
    k_mg_sub_mean<<<grid_for(n), PT, 0, st>>>(v, n, b.scalar);
}

static void vcycle(const MgPlan& p, int l, const MgBuffers& b, cudaStream_t st)
{
    const int nx = p.dim[l][0], ny = p.dim[l][1], nz = p.dim[l][2];
    const int64_t n = (int64_t)nx * ny * nz;
    if (l == p.levels - 1) {  // coarsest: zero-mean right-hand side, many sweeps
        sub_mean(b.f + p.off[l], n, b, st);
        const int m = std::max(nx, std::max(ny, nz));
        smooth(p, l, b, std::max(8, 2 * m * m), st);
        return;
    }
    smooth(p, l, b, 2, st);
    k_mg_residual<<<grid_for(n), PT, 0, st>>>(b.phi + p.off[l], b.f + p.off[l], b.r + p.off[l], nx, ny, nz);
    const int64_t nc = (int64_t)p.dim[l + 1][0] * p.dim[l + 1][1] * p.dim[l + 1][2];
    k_mg_restrict<<<grid_for(nc), PT, 0, st>>>(b.r + p.off[l], b.f + p.off[l + 1], nx, ny, nz);
    cudaMemsetAsync(b.phi + p.off[l + 1], 0, sizeof(double) * nc, st);
    vcycle(p, l + 1, b, st);
    k_mg_prolong<<<grid_for(n), PT, 0, st>>>(b.phi + p.off[l + 1], b.phi + p.off[l], nx, ny, nz);
    smooth(p, l, b, 2, st);
}

int64_t mg_cycle_kernels(const MgPlan& p)
{
    int64_t k = 0;
    for (int l = 0; l < p.levels - 1; ++l) k += 4 + 1 + 1 + 1 + 4;  // smooth, residual, restrict, prolong, smooth
    const int l = p.levels - 1;
    const int m = std::max(p.dim[l][0], std::max(p.dim[l][1], p.dim[l][2]));
    return k + 3 + 2 * (int64_t)std::max(8, 2 * m * m);  // coarsest: mean, sweeps
}

cudaError_t elec_solve(const RepDesc& D, const VacRec* recs, const int32_t* counts, int cap, int64_t n_vac,
                       double q, double scale, int cycles, const MgPlan& p, const MgBuffers& b, double* resid_rel,
                       cudaStream_t st)
{
    const int64_t n = p.dim[0][0] * (int64_t)p.dim[0][1] * p.dim[0][2];
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * n, st);
    if (e != cudaSuccess) return e;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    k_mg_deposit<<<grid_for(nfrag * cap), PT, 0, st>>>(D, recs, counts, cap, b.cnt);
    k_mg_rhs<<<grid_for(n), PT, 0, st>>>(b.cnt, n, 0.5 * q, q * (double)n_vac / (double)n, scale, b.f);
    e = cudaMemsetAsync(b.phi, 0, sizeof(double) * n, st);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < cycles; ++c) vcycle(p, 0, b, st);
    sub_mean(b.phi, n, b, st);
    if (resid_rel) {  // max |f - A phi| / max |f|
        k_mg_residual<<<grid_for(n), PT, 0, st>>>(b.phi, b.f, b.r, p.dim[0][0], p.dim[0][1], p.dim[0][2]);
        k_mg_partial<<<MG_PARTIALS, PT, 0, st>>>(b.r, n, b.part, 1);
        k_mg_final<<<1, 32, 0, st>>>(b.part, MG_PARTIALS, b.scalar, 1);
        k_mg_partial<<<MG_PARTIALS, PT, 0, st>>>(b.f, n, b.part, 1);
        k_mg_final<<<1, 32, 0, st>>>(b.part, MG_PARTIALS, b.scalar + 1, 1);
        double h[2];
        e = cudaMemcpyAsync(h, b.scalar, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        *resid_rel = h[1] > 0.0 ? h[0] / h[1] : 0.0;
    }
    return cudaGetLastError();
}

cudaError_t elec_solve_unit(const RepDesc& D, int t, double scale, int cycles, const MgPlan& p, const MgBuffers& b,
                            cudaStream_t st)
{
    // one unit charge (q = 1) on the mid-lattice site of type t: two half-charges
    const int nx = D.L[0], ny = D.L[1], nz = D.L[2];
    const int64_t n = (int64_t)nx * ny * nz;
    std::vector<int32_t> cnt((size_t)n, 0);
    const int x = nx / 2, y = ny / 2, z = nz / 2;
    cnt[((size_t)z * ny + y) * nx + x] += 1;
    cnt[((size_t)((z + (t == 2)) % nz) * ny + (y + (t == 1)) % ny) * nx + (x + (t == 0)) % nx] += 1;
    cudaError_t e = cudaMemcpyAsync(b.cnt, cnt.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_mg_rhs<<<grid_for(n), PT, 0, st>>>(b.cnt, n, 0.5, 1.0 / (double)n, scale, b.f);
    e = cudaMemsetAsync(b.phi, 0, sizeof(double) * n, st);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < cycles; ++c) vcycle(p, 0, b, st);
    sub_mean(b.phi, n, b, st);
    e = cudaStreamSynchronize(st);  // the caller reads b.phi next (host copy in the same stream)
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t elec_update(const RepDesc& D, const double* phi, double q, int32_t* u, int32_t* field, unsigned* umax,
                        cudaStream_t st)
{
    k_elec_update<<<grid_for(D.nsite), PT, 0, st>>>(D, phi, q, u, field, umax);
    return cudaGetLastError();
}

cudaError_t elec_add(int32_t* field, const int32_t* u, int64_t n, cudaStream_t st)
{
    k_elec_add<<<grid_for(n), PT, 0, st>>>(field, u, n);
    return cudaGetLastError();
}

}  // namespace fkmc
