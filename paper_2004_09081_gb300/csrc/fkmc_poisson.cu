// fkmc_poisson.cu -- electrostatic potential of the vacancy charges for the
// mu-scale model of arXiv:2004.09081 (Sec. "Oxygen diffusion in mu-scale
// BaTiO3 model": the potential comes from a Poisson equation).  The source is
// read as the vacancies' own charge q e, split in halves between the two B
// nodes (cell corners) of each vacancy's O-site bond, against a uniform
// background; the grid is periodic with spacing a:
//
//     6 phi(n) - sum_{6 neighbours} phi(n') = Q(n) / (eps0 eps_r a)        [V]
//
// solved by defect correction in FP64 around geometric multigrid V-cycles in
// FP32 (vertex-centred coarsening by 2 while every dimension is even;
// red-black Gauss-Seidel where all dimensions of a level are even, damped
// Jacobi otherwise and on the coarsest level; full-weighting restriction,
// trilinear prolongation).  Every reduction is
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

// The level-by-level stencil kernels run on 3-D grids: blockIdx.y / blockIdx.z
// are the row (y, z), threads walk x; all index arithmetic is 32-bit.  They are
// templates over the number type: the V-cycle runs in FP32 (below, the FP64
// defect correction around it), the final residual check in FP64.
constexpr int XT = 128;
constexpr double SIXTH = 1.0 / 6.0;

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ T nb_sum(const T* v, int x, int y, int z, int nx, int ny, int nz)
{
    const int row = (z * ny + y) * nx;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    T s = v[row + xm];
    s = add_rn(s, v[row + xp]);
    s = add_rn(s, v[(z * ny + ym) * nx + x]);
    s = add_rn(s, v[(z * ny + yp) * nx + x]);
    s = add_rn(s, v[(zm * ny + y) * nx + x]);
    s = add_rn(s, v[(zp * ny + y) * nx + x]);
    return s;
}

// red-black Gauss-Seidel half-sweep over the nodes of one colour (all
// dimensions even: the colouring is consistent across the periodic seams);
// thread k of a row takes x = 2k + the row's colour offset
template <typename T>
__global__ void __launch_bounds__(XT) k_mg_rb(T* phi, const T* f, int nx, int ny, int nz, int colour)
{
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = 2 * (blockIdx.x * XT + threadIdx.x) + ((y + z + colour) & 1);
    if (x >= nx) return;
    const int i = (z * ny + y) * nx + x;
    phi[i] = mul_rn(add_rn(f[i], nb_sum(phi, x, y, z, nx, ny, nz)), (T)SIXTH);
}

// damped Jacobi sweep, out = (1-w) in + w (f + sum nb) / 6
template <typename T>
__global__ void __launch_bounds__(XT) k_mg_jacobi(const T* in, T* out, const T* f, int nx, int ny, int nz, T w)
{
    const int y = blockIdx.y, z = blockIdx.z, x = blockIdx.x * XT + threadIdx.x;
    if (x >= nx) return;
    const int i = (z * ny + y) * nx + x;
    const T gs = mul_rn(add_rn(f[i], nb_sum(in, x, y, z, nx, ny, nz)), (T)SIXTH);
    out[i] = add_rn(mul_rn((T)1 - w, in[i]), mul_rn(w, gs));
}

// r = f - A phi
template <typename T>
__global__ void __launch_bounds__(XT) k_mg_residual(const T* phi, const T* f, T* r, int nx, int ny, int nz)
{
    const int y = blockIdx.y, z = blockIdx.z, x = blockIdx.x * XT + threadIdx.x;
    if (x >= nx) return;
    const int i = (z * ny + y) * nx + x;
    r[i] = add_rn(f[i], -add_rn(mul_rn((T)6, phi[i]), -nb_sum(phi, x, y, z, nx, ny, nz)));
}

// the defect of the FP64 potential, d = f - A phi in FP64, rounded to FP32: the
// right-hand side of the FP32 correction cycle
__global__ void __launch_bounds__(XT) k_mg_defect(const double* phi, const double* f, float* d, int nx, int ny,
                                                   int nz)
{
    const int y = blockIdx.y, z = blockIdx.z, x = blockIdx.x * XT + threadIdx.x;
    if (x >= nx) return;
    const int i = (z * ny + y) * nx + x;
    d[i] = __double2float_rn(__dadd_rn(f[i], -__dadd_rn(__dmul_rn(6.0, phi[i]), -nb_sum(phi, x, y, z, nx, ny, nz))));
}

// phi += e (the FP32 correction, converted exactly)
__global__ void k_mg_correct(double* phi, const float* e, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        phi[i] = __dadd_rn(phi[i], (double)e[i]);
}

// coarse f = 4 x full weighting of the fine residual (weights (1,2,1)^3 / 64);
// the grid covers the coarse level
template <typename T>
__global__ void __launch_bounds__(XT) k_mg_restrict(const T* r, T* fc, int nx, int ny, int nz)
{
    const int cx = nx / 2, cy = ny / 2;
    const int Y = blockIdx.y, Z = blockIdx.z, X = blockIdx.x * XT + threadIdx.x;
    if (X >= cx) return;
    T s = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        const int zz = wrap_(2 * Z + dz, nz);
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = wrap_(2 * Y + dy, ny);
            const T* row = r + (zz * ny + yy) * nx;
            const T wr = (T)((2 - (dz != 0)) * (2 - (dy != 0)));
            const T line = add_rn(add_rn(row[wrap_(2 * X - 1, nx)], mul_rn((T)2, row[2 * X])), row[wrap_(2 * X + 1, nx)]);
            s = add_rn(s, mul_rn(wr, line));
        }
    }
    fc[(Z * cy + Y) * cx + X] = mul_rn(s, (T)(4.0 / 64.0));
}

// phi_fine += trilinear interpolation of the coarse correction
template <typename T>
__global__ void __launch_bounds__(XT) k_mg_prolong(const T* ec, T* phi, int nx, int ny, int nz)
{
    const int y = blockIdx.y, z = blockIdx.z, x = blockIdx.x * XT + threadIdx.x;
    if (x >= nx) return;
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int X = x >> 1, Y = y >> 1, Z = z >> 1, ox = x & 1, oy = y & 1, oz = z & 1;
    T s = 0;
    for (int dz = 0; dz <= oz; ++dz)
        for (int dy = 0; dy <= oy; ++dy)
            for (int dx = 0; dx <= ox; ++dx)
                s = add_rn(s, ec[(wrap_(Z + dz, cz) * cy + wrap_(Y + dy, cy)) * cx + wrap_(X + dx, cx)]);
    const int i = (z * ny + y) * nx + x;
    phi[i] = add_rn(phi[i], mul_rn(s, (T)(1.0 / (double)(1 << (ox + oy + oz)))));
}

// deterministic sum (or max |v|) in FP64: per-block partials (fixed grid), then
// one thread in order
template <typename T>
__global__ void k_mg_partial(const T* v, int64_t n, double* part, int absmax)
{
    __shared__ double sh[PT];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * PT + threadIdx.x; i < n; i += (int64_t)gridDim.x * PT)
        s = absmax ? fmax(s, fabs((double)v[i])) : __dadd_rn(s, (double)v[i]);
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
template <typename T>
__global__ void k_mg_sub_mean(T* v, int64_t n, const double* sum)
{
    const T m = (T)__ddiv_rn(*sum, (double)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = add_rn(v[i], -m);
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


// ---- the small levels of a V-cycle in one block: levels ls .. coarsest live
// in shared memory (phi, f and scratch of each level, at most SMALL_BYTES), the
// same operations as the level-by-level kernels separated by __syncthreads.
// The block reads the iterate and right-hand side of level ls from global
// memory and writes back the iterate after the sub-cycle.  Node coordinates
// come from exact multiply-high division: for 2 <= d and i, d < 2^16,
// floor(i / d) = umulhi(i, ceil(2^32 / d)) (the rounding excess of the
// reciprocal, times i, stays below 2^32).
constexpr int SMALL_BYTES = 200 * 1024;
constexpr int ST = 1024;

struct SmallLevels {
    int ls, levels;
    int dim[MG_MAX_LEVELS][3];
    unsigned rx[MG_MAX_LEVELS], ry[MG_MAX_LEVELS];  // ceil(2^32 / nx), ceil(2^32 / ny)
    int offs[MG_MAX_LEVELS];  // node offset of each level in the shared arrays
    int nodes;                // shared nodes per array
    int64_t off_ls;           // global offset of level ls
    int coarse_sweeps;
};

__device__ __forceinline__ void s_coords(const SmallLevels& P, int l, int i, int& x, int& y, int& z)
{
    const int nx = P.dim[l][0], ny = P.dim[l][1];
    const int q = (int)__umulhi((unsigned)i, P.rx[l]);
    x = i - q * nx;
    z = (int)__umulhi((unsigned)q, P.ry[l]);
    y = q - z * ny;
}

template <typename T>
__device__ __forceinline__ T s_nb(const T* v, int x, int y, int z, int nx, int ny, int nz)
{
    T s = v[nidx(wrap_(x - 1, nx), y, z, nx, ny)];
    s = add_rn(s, v[nidx(wrap_(x + 1, nx), y, z, nx, ny)]);
    s = add_rn(s, v[nidx(x, wrap_(y - 1, ny), z, nx, ny)]);
    s = add_rn(s, v[nidx(x, wrap_(y + 1, ny), z, nx, ny)]);
    s = add_rn(s, v[nidx(x, y, wrap_(z - 1, nz), nx, ny)]);
    s = add_rn(s, v[nidx(x, y, wrap_(z + 1, nz), nx, ny)]);
    return s;
}

template <typename T>
__device__ void s_smooth(const SmallLevels& P, int l, T* phi, const T* f, T* tmp, int sweeps)
{
    const int nx = P.dim[l][0], ny = P.dim[l][1], nz = P.dim[l][2];
    const int n = nx * ny * nz;
    const bool even = nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0;
    const T w = (T)(6.0 / 7.0);
    for (int k = 0; k < sweeps; ++k) {
        for (int half = 0; half < 2; ++half) {
            const T* in = even ? phi : (half == 0 ? phi : tmp);
            T* out = even ? phi : (half == 0 ? tmp : phi);
            for (int i = threadIdx.x; i < n; i += ST) {
                int x, y, z;
                s_coords(P, l, i, x, y, z);
                if (even && ((x + y + z) & 1) != half) continue;
                const T gs = mul_rn(add_rn(f[i], s_nb(in, x, y, z, nx, ny, nz)), (T)SIXTH);
                out[i] = even ? gs : add_rn(mul_rn((T)1 - w, in[i]), mul_rn(w, gs));
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(ST) k_mg_small(SmallLevels P, T* phi_g, const T* f_g)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    T* phi_all = reinterpret_cast<T*>(s_raw);
    T* f_all = phi_all + P.nodes;
    T* r_all = phi_all + 2 * P.nodes;
    __shared__ double red[ST];
    const int last = P.levels - 1;
    {
        const int n0 = P.dim[P.ls][0] * P.dim[P.ls][1] * P.dim[P.ls][2];
        for (int i = threadIdx.x; i < n0; i += ST) {
            phi_all[i] = phi_g[P.off_ls + i];  // the iterate so far (zero below the finest level)
            f_all[i] = f_g[P.off_ls + i];
        }
        __syncthreads();
    }
    for (int l = P.ls; l < last; ++l) {  // down: pre-smooth, residual, restrict
        const int nx = P.dim[l][0], ny = P.dim[l][1], nz = P.dim[l][2];
        const int n = nx * ny * nz;
        T* phi = phi_all + P.offs[l];
        const T* f = f_all + P.offs[l];
        T* r = r_all + P.offs[l];
        s_smooth(P, l, phi, f, r, 2);
        for (int i = threadIdx.x; i < n; i += ST) {
            int x, y, z;
            s_coords(P, l, i, x, y, z);
            r[i] = add_rn(f[i], -add_rn(mul_rn((T)6, phi[i]), -s_nb(phi, x, y, z, nx, ny, nz)));
        }
        __syncthreads();
        const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
        T* fc = f_all + P.offs[l + 1];
        T* pc = phi_all + P.offs[l + 1];
        for (int i = threadIdx.x; i < cx * cy * cz; i += ST) {
            int X, Y, Z;
            s_coords(P, l + 1, i, X, Y, Z);
            T s = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const T w = (T)((2 - (dx != 0)) * (2 - (dy != 0)) * (2 - (dz != 0)));
                        s = add_rn(s, mul_rn(w, r[nidx(wrap_(2 * X + dx, nx), wrap_(2 * Y + dy, ny),
                                                       wrap_(2 * Z + dz, nz), nx, ny)]));
                    }
            fc[i] = mul_rn(s, (T)(4.0 / 64.0));
            pc[i] = 0;
        }
        __syncthreads();
    }
    {  // coarsest: zero-mean right-hand side (block tree sum in FP64, fixed order), sweeps
        const int n = P.dim[last][0] * P.dim[last][1] * P.dim[last][2];
        T* f = f_all + P.offs[last];
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += ST) s = __dadd_rn(s, (double)f[i]);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = ST / 2; w; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
            __syncthreads();
        }
        const T m = (T)__ddiv_rn(red[0], (double)n);
        for (int i = threadIdx.x; i < n; i += ST) f[i] = add_rn(f[i], -m);
        __syncthreads();
        s_smooth(P, last, phi_all + P.offs[last], (const T*)f, r_all + P.offs[last], P.coarse_sweeps);
    }
    for (int l = last - 1; l >= P.ls; --l) {  // up: prolong, post-smooth
        const int nx = P.dim[l][0], ny = P.dim[l][1];
        const int n = nx * ny * P.dim[l][2], cx = nx / 2, cy = ny / 2, cz = P.dim[l][2] / 2;
        T* phi = phi_all + P.offs[l];
        const T* ec = phi_all + P.offs[l + 1];
        for (int i = threadIdx.x; i < n; i += ST) {
            int x, y, z;
            s_coords(P, l, i, x, y, z);
            const int X = x >> 1, Y = y >> 1, Z = z >> 1, ox = x & 1, oy = y & 1, oz = z & 1;
            T s = 0;
            for (int dz = 0; dz <= oz; ++dz)
                for (int dy = 0; dy <= oy; ++dy)
                    for (int dx = 0; dx <= ox; ++dx)
                        s = add_rn(s, ec[nidx(wrap_(X + dx, cx), wrap_(Y + dy, cy), wrap_(Z + dz, cz), cx, cy)]);
            phi[i] = add_rn(phi[i], mul_rn(s, (T)(1.0 / (double)(1 << (ox + oy + oz)))));
        }
        __syncthreads();
        s_smooth(P, l, phi, (const T*)(f_all + P.offs[l]), r_all + P.offs[l], 2);
    }
    const int n0 = P.dim[P.ls][0] * P.dim[P.ls][1] * P.dim[P.ls][2];
    for (int i = threadIdx.x; i < n0; i += ST) phi_g[P.off_ls + i] = phi_all[i];
}

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

static dim3 rows(int nx_threads, int ny, int nz) { return dim3((unsigned)((nx_threads + XT - 1) / XT), ny, nz); }

// `sweeps` smoothing sweeps of level l on the level-stacked arrays u (iterate), f
// and tmp (Jacobi scratch)
template <typename T>
static void smooth(const MgPlan& p, int l, T* u, const T* f, T* tmp, int sweeps, cudaStream_t st)
{
    const int nx = p.dim[l][0], ny = p.dim[l][1], nz = p.dim[l][2];
    u += p.off[l];
    f += p.off[l];
    tmp += p.off[l];
    for (int k = 0; k < sweeps; ++k) {
        if (level_even(p, l)) {
            k_mg_rb<T><<<rows(nx / 2, ny, nz), XT, 0, st>>>(u, f, nx, ny, nz, 0);
            k_mg_rb<T><<<rows(nx / 2, ny, nz), XT, 0, st>>>(u, f, nx, ny, nz, 1);
        } else {  // two Jacobi half-steps through the scratch level buffer
            k_mg_jacobi<T><<<rows(nx, ny, nz), XT, 0, st>>>(u, tmp, f, nx, ny, nz, (T)(6.0 / 7.0));
            k_mg_jacobi<T><<<rows(nx, ny, nz), XT, 0, st>>>(tmp, u, f, nx, ny, nz, (T)(6.0 / 7.0));
        }
    }
}

template <typename T>
static void sub_mean(T* v, int64_t n, const MgBuffers& b, cudaStream_t st)
{
    k_mg_partial<T><<<MG_PARTIALS, PT, 0, st>>>(v, n, b.part, 0);
    k_mg_final<<<1, 32, 0, st>>>(b.part, MG_PARTIALS, b.scalar, 0);
    k_mg_sub_mean<T><<<grid_for(n), PT, 0, st>>>(v, n, b.scalar);
}

static int coarse_sweeps(const MgPlan& p)
{
    const int l = p.levels - 1;
    const int m = std::max(p.dim[l][0], std::max(p.dim[l][1], p.dim[l][2]));
    return std::max(8, 2 * m * m);
}

// first level from which all coarser levels fit one block's shared memory
// (iterate, right-hand side and scratch: 12 bytes per node in FP32), or levels
static int first_small(const MgPlan& p)
{
    int ls = p.levels;
    int64_t nodes = 0;
    while (ls > 0) {
        const int* d = p.dim[ls - 1];
        const int64_t n = (int64_t)d[0] * d[1] * d[2];
        if (3 * (int64_t)sizeof(float) * (nodes + n) > SMALL_BYTES || d[0] < 2 || d[1] < 2) break;
        nodes += n;
        --ls;
    }
    return ls;
}

// one V-cycle from level l on the level-stacked FP32 arrays: u the iterate
// (correction), f the right-hand side, r the residual / scratch
static void vcycle(const MgPlan& p, int l, float* u, float* f, float* r, const MgBuffers& b, cudaStream_t st)
{
    const int nx = p.dim[l][0], ny = p.dim[l][1], nz = p.dim[l][2];
    const int64_t n = (int64_t)nx * ny * nz;
    if (l == first_small(p)) {  // the rest of the cycle in one block, in shared memory
        SmallLevels P{};
        P.ls = l;
        P.levels = p.levels;
        int nodes = 0;
        for (int k = 0; k < p.levels; ++k) {
            for (int d = 0; d < 3; ++d) P.dim[k][d] = p.dim[k][d];
            if (k >= l) {
                P.offs[k] = nodes;
                nodes += p.dim[k][0] * p.dim[k][1] * p.dim[k][2];
                P.rx[k] = (unsigned)(((1ull << 32) + p.dim[k][0] - 1) / p.dim[k][0]);
                P.ry[k] = (unsigned)(((1ull << 32) + p.dim[k][1] - 1) / p.dim[k][1]);
            }
        }
        P.nodes = nodes;
        P.off_ls = p.off[l];
        P.coarse_sweeps = coarse_sweeps(p);
        const size_t bytes = sizeof(float) * 3 * (size_t)nodes;
        static bool opted[64] = {};  // the shared-memory opt-in, once per device
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !opted[dev]) {
            cudaFuncSetAttribute(k_mg_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMALL_BYTES);
            opted[dev] = true;
        }
        k_mg_small<float><<<1, ST, bytes, st>>>(P, u, f);
        return;
    }
    if (l == p.levels - 1) {  // coarsest: zero-mean right-hand side, many sweeps
        sub_mean(f + p.off[l], n, b, st);
        smooth(p, l, u, f, r, coarse_sweeps(p), st);
        return;
    }
    smooth(p, l, u, f, r, 2, st);
    k_mg_residual<float><<<rows(nx, ny, nz), XT, 0, st>>>(u + p.off[l], f + p.off[l], r + p.off[l], nx, ny, nz);
    const int64_t nc = (int64_t)p.dim[l + 1][0] * p.dim[l + 1][1] * p.dim[l + 1][2];
    k_mg_restrict<float><<<rows(nx / 2, ny / 2, nz / 2), XT, 0, st>>>(r + p.off[l], f + p.off[l + 1], nx, ny, nz);
    cudaMemsetAsync(u + p.off[l + 1], 0, sizeof(float) * nc, st);
    vcycle(p, l + 1, u, f, r, b, st);
    k_mg_prolong<float><<<rows(nx, ny, nz), XT, 0, st>>>(u + p.off[l + 1], u + p.off[l], nx, ny, nz);
    smooth(p, l, u, f, r, 2, st);
}

// One cycle of defect correction: the FP64 defect of phi, one FP32 V-cycle on
// the correction equation A e = d from e = 0, phi += e.  Each cycle removes the
// same share of the error as an FP64 V-cycle (the FP32 rounding is relative to
// the current defect), so the iteration still converges to FP64 accuracy, and
// only the fine-level defect and update use the FP64 pipe.
static void mixed_cycle(const MgPlan& p, const MgBuffers& b, cudaStream_t st)
{
    const int nx = p.dim[0][0], ny = p.dim[0][1], nz = p.dim[0][2];
    const int64_t n = (int64_t)nx * ny * nz;
    k_mg_defect<<<rows(nx, ny, nz), XT, 0, st>>>(b.phi, b.f, b.g, nx, ny, nz);
    cudaMemsetAsync(b.e, 0, sizeof(float) * n, st);
    vcycle(p, 0, b.e, b.g, b.s, b, st);
    k_mg_correct<<<grid_for(n), PT, 0, st>>>(b.phi, b.e, n);
}

int64_t mg_cycle_kernels(const MgPlan& p)
{
    const int ls = first_small(p);
    int64_t k = 2;                                                               // defect, correction
    for (int l = 0; l < std::min(ls, p.levels - 1); ++l) k += 4 + 1 + 1 + 1 + 4;  // smooth, residual, restrict,
                                                                                 // prolong, smooth
    if (ls < p.levels) return k + 1;                                            // the one-block rest
    return k + 3 + 2 * (int64_t)coarse_sweeps(p);                               // coarsest: mean, sweeps
}

cudaError_t elec_solve(const RepDesc& D, const VacRec* recs, const int32_t* counts, int cap, int64_t n_vac,
                       double q, double scale, int cycles, const MgPlan& p, const MgBuffers& b, double* resid_rel,
                       const double* init, double* save, cudaStream_t st)
{
    const int64_t n = p.dim[0][0] * (int64_t)p.dim[0][1] * p.dim[0][2];
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * n, st);
    if (e != cudaSuccess) return e;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    k_mg_deposit<<<grid_for(nfrag * cap), PT, 0, st>>>(D, recs, counts, cap, b.cnt);
    k_mg_rhs<<<grid_for(n), PT, 0, st>>>(b.cnt, n, 0.5 * q, q * (double)n_vac / (double)n, scale, b.f);
    e = init ? cudaMemcpyAsync(b.phi, init, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)
             : cudaMemsetAsync(b.phi, 0, sizeof(double) * n, st);  // warm start from the last solve
    if (e != cudaSuccess) return e;
    for (int c = 0; c < cycles; ++c) mixed_cycle(p, b, st);
    sub_mean(b.phi, n, b, st);
    if (save) {
        e = cudaMemcpyAsync(save, b.phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (resid_rel) {  // max |f - A phi| / max |f|, all in FP64
        k_mg_residual<double><<<rows(p.dim[0][0], p.dim[0][1], p.dim[0][2]), XT, 0, st>>>(
            b.phi, b.f, b.r, p.dim[0][0], p.dim[0][1], p.dim[0][2]);
        k_mg_partial<double><<<MG_PARTIALS, PT, 0, st>>>(b.r, n, b.part, 1);
        k_mg_final<<<1, 32, 0, st>>>(b.part, MG_PARTIALS, b.scalar, 1);
        k_mg_partial<double><<<MG_PARTIALS, PT, 0, st>>>(b.f, n, b.part, 1);
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
    for (int c = 0; c < cycles; ++c) mixed_cycle(p, b, st);
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
