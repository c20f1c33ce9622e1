// Kernels of the collision operator, templated on the real type T.
//
// Data flow of one evaluation (Algorithm 1, Sec. 3.4, with the transform
// pairs of each product cancelled by linearity):
//   forward : ghat = DFT(f) / N^d                          (Eq. (3.1))
//   pass 1  : per shifted field x and plane j1, the weighted spectrum
//             ghat_j exp(-i pi j.x / L) (separable per axis) and its inverse
//             transform over the trailing d-1 axes     -> H[field][j1][plane]
//   pass 2  : per column of the trailing axes, the inverse transform along
//             axis 0 of C, A, B; then W_p [A B (C + F) - C F (A + B)]
//             accumulated per quadrature group           -> Qacc[group]
//   finalize: Q = 2^{1-d} sum over groups of Qacc         (real part of K)
// Grids are row-major, last axis fastest; P = N^{d-1} columns per plane.
#pragma once

#include <cstdint>

#include "wke_check.cuh"
#include "wke_fft.cuh"
#include "wke_internal.h"

namespace wke {

// ------------------------------------------------------------------ helpers
template <typename T> struct KCfg {
    // warps per block of the column / row kernels
    static constexpr int WARPS = 8;
};

template <int N> struct Work {
    static constexpr int PITCH = N + 4;   // = 4 (mod 16) for N a multiple of 16
};

template <typename T, int N> __host__ __device__ constexpr size_t scratch_elems_per_warp() {
    return (size_t)LineCfg<T, N>::LPW * LinePad<N>::PITCH;
}

// Asynchronous global -> shared copy of one complex value (cp.async); the
// issuing thread later reads the same slot after cp.async.wait_group.
template <typename T> __device__ __forceinline__ void cp_async_cx(cx<T> *dst, const cx<T> *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(cx<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes global -> shared, both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

template <typename T, int N>
__device__ __forceinline__ void load_twiddles(cx<T> *tw, const cx<T> *tw_g) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();
}
// The same in two steps: the global load issued first, so that it is in
// flight together with a kernel's own first loads, and the shared-memory
// store and barrier once those are issued.
template <typename T, int N> __device__ __forceinline__ cx<T> twiddle_fetch(const cx<T> *tw_g) {
    return threadIdx.x < N ? tw_g[threadIdx.x] : mkc<T>((T)0, (T)0);
}
template <typename T, int N>
__device__ __forceinline__ void twiddle_store(cx<T> *tw, cx<T> mine, const cx<T> *tw_g) {
    if (threadIdx.x < N) tw[threadIdx.x] = mine;
    for (int i = threadIdx.x + blockDim.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();
}

// ------------------------------------------------------------------ forward
// The forward transform computes in TC: double (the default) or, on request
// for FP32 plans, float.
// 3D: forward transform along axis 1 of every (i1, i3) line, in place (the
// rows were transformed by k_fwd_rows_2d over all N^2 rows).  A warp holds
// LPW lines of consecutive i3.  The rows of a real f are Hermitian in j3, so
// only the columns j3 = 0 .. N/2 are transformed (N (N/2 + 1) lines); the
// axis-0 pass writes the other half of the coefficients by symmetry.
template <int N, typename TC = double>
__global__ void k_fwd_mid_3d(cx<TC> *__restrict__ tmp, const cx<TC> *__restrict__ tw_g) {
    typedef FwdCfg<TC, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<TC> *tw = reinterpret_cast<cx<TC> *>(smem_raw);
    cx<TC> *scratch = tw + N;
    load_twiddles<TC, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    constexpr int H = N / 2 + 1;
    const int line = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    const int i1 = line / H, i3 = line - i1 * H;
    cx<TC> *base = tmp + (size_t)i1 * N * N + i3;
    cx<TC> *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    cx<TC> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = base[(size_t)(t + e * TPL) * N];
    line_fft<TC, N, E, -1>(v, t, scr, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) base[(size_t)(t + e * TPL) * N] = v[e];
}

// Forward transform of every row (the last axis): the N rows of a 2D grid,
// or the N^2 rows of a 3D one.  PACK: each line transforms two real rows at
// once, Z = DFT(f_a + i f_b), and separates them with the partner value
// Z(N - j) from the lane holding it (f_a and f_b are real, so
// F_a(j) = (Z(j) + conj Z(N - j)) / 2 and F_b(j) = (Z(j) - conj Z(N - j)) / 2i):
// half the transforms.  Thread t of a line holds j = t + e TPL, so Z(N - j)
// sits in thread TPL - t at e' = E - 1 - e (thread 0: itself, e' = E - e mod E).
template <typename TIn, int N, typename TC = double, bool PACK = false>
__global__ void k_fwd_rows_2d(const TIn *__restrict__ f, cx<TC> *__restrict__ tmp, const cx<TC> *__restrict__ tw_g) {
    typedef FwdCfg<TC, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<TC> *tw = reinterpret_cast<cx<TC> *>(smem_raw);
    cx<TC> *scratch = tw + N;
    load_twiddles<TC, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    const int i1 = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    cx<TC> *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    cx<TC> v[E];
    if constexpr (PACK) {
        const size_t ra = (size_t)(2 * i1) * N, rb = ra + N;     // rows 2 i1 and 2 i1 + 1
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = mkc<TC>((TC)f[ra + t + e * TPL], (TC)f[rb + t + e * TPL]);
        line_fft<TC, N, E, -1>(v, t, scr, tw);
        const int partner = ((TPL - t) % TPL) * LPW + c;
        cx<TC> zr[E];   // Z(N - j) for this thread's j = t + e TPL
#pragma unroll
        for (int es = 0; es < E; ++es) {
            const cx<TC> w = mkc<TC>(__shfl_sync(0xffffffffu, v[es].x, partner),
                                     __shfl_sync(0xffffffffu, v[es].y, partner));
            if (t == 0)
                zr[(E - es) % E] = w;
            else
                zr[E - 1 - es] = w;
        }
        const TC h = (TC)0.5;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const cx<TC> z = v[e], m = zr[e];
            tmp[ra + t + e * TPL] = mkc<TC>(h * (z.x + m.x), h * (z.y - m.y));
            tmp[rb + t + e * TPL] = mkc<TC>(h * (z.y + m.y), h * (m.x - z.x));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = mkc<TC>((TC)f[(size_t)i1 * N + t + e * TPL], (TC)0);
        line_fft<TC, N, E, -1>(v, t, scr, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) tmp[(size_t)i1 * N + t + e * TPL] = v[e];
    }
}

// Both d: forward transform along axis 0 of every column; writes
// ghat = DFT / N^d in T, optionally zeroing modes with a component -N/2.
// When `nslice` is not null it also receives the Nyquist slices used by the
// Nyquist tables: slice ax holds the modes with j_ax = -N/2 (position N/2),
// indexed by the other axes in increasing order, with the modes that have an
// earlier axis at -N/2 set to zero (so the slices are disjoint).
// HALF (3D, after k_fwd_mid_3d): only the columns (j2, j3 <= N/2) are
// transformed, and each coefficient with 0 < j3 < N/2 also gives its partner
// ghat(-j) = conj ghat(j) (f is real).
template <typename TOut, int N, typename TC = double, bool HALF = false>
__global__ void k_fwd_cols(const cx<TC> *__restrict__ tmp, cx<TOut> *__restrict__ ghat,
                           const cx<TC> *__restrict__ tw_g, int P, int d, double inv_nd, int nyq_zero,
                           cx<TOut> *__restrict__ nslice) {
    typedef FwdCfg<TC, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<TC> *tw = reinterpret_cast<cx<TC> *>(smem_raw);
    cx<TC> *scratch = tw + N;
    load_twiddles<TC, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    const int line = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    cx<TC> *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    cx<TC> v[E];
    if constexpr (HALF) {
        constexpr int H = N / 2 + 1, H2 = N / 2;
        const int j2 = line / H, j3 = line - j2 * H;
        const int col = j2 * N + j3;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = tmp[(size_t)(t + e * TPL) * P + col];
        line_fft<TC, N, E, -1>(v, t, scr, tw);
        const cx<TOut> zero = mkc<TOut>((TOut)0, (TOut)0);
        auto emit = [&](int a1, int a2, int a3, cx<TC> x) {
            if (nyq_zero && (a1 == H2 || a2 == H2 || a3 == H2)) x = mkc<TC>((TC)0, (TC)0);
            const cx<TOut> val = mkc<TOut>((TOut)(x.x * (TC)inv_nd), (TOut)(x.y * (TC)inv_nd));
            ghat[(size_t)a1 * P + a2 * N + a3] = val;
            if (nslice) {
                if (a1 == H2) nslice[(size_t)a2 * N + a3] = val;
                if (a2 == H2) nslice[(size_t)N * N + (size_t)a1 * N + a3] = a1 == H2 ? zero : val;
                if (a3 == H2) nslice[(size_t)2 * N * N + (size_t)a1 * N + a2] = (a1 == H2 || a2 == H2) ? zero : val;
            }
        };
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j1 = t + e * TPL;
            emit(j1, j2, j3, v[e]);
            if (j3 > 0 && j3 < H2) emit((N - j1) % N, (N - j2) % N, N - j3, mkc<TC>(v[e].x, -v[e].y));
        }
    } else {
        const int col = line;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = tmp[(size_t)(t + e * TPL) * P + col];
        line_fft<TC, N, E, -1>(v, t, scr, tw);
        bool col_nyq = false;
        if (nyq_zero) {
            int rest = col;
            for (int a = 1; a < d; ++a) {
                if (rest % N == N / 2) col_nyq = true;
                rest /= N;
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j1 = t + e * TPL;
            cx<TC> x = v[e];
            if (nyq_zero && (col_nyq || j1 == N / 2)) x = mkc<TC>((TC)0, (TC)0);
            const cx<TOut> val = mkc<TOut>((TOut)(x.x * (TC)inv_nd), (TOut)(x.y * (TC)inv_nd));
            ghat[(size_t)j1 * P + col] = val;
            if (nslice) {
                const cx<TOut> zero = mkc<TOut>((TOut)0, (TOut)0);
                constexpr int H2 = N / 2;
                if (d == 3) {
                    const int j2 = col / N, j3 = col - j2 * N;
                    if (j1 == H2) nslice[(size_t)j2 * N + j3] = val;
                    if (j2 == H2) nslice[(size_t)N * N + (size_t)j1 * N + j3] = j1 == H2 ? zero : val;
                    if (j3 == H2) nslice[(size_t)2 * N * N + (size_t)j1 * N + j2] = (j1 == H2 || j2 == H2) ? zero : val;
                } else {
                    if (j1 == H2) nslice[col] = val;
                    if (col == H2) nslice[N + j1] = j1 == H2 ? zero : val;
                }
            }
        }
    }
}

// Q-hat: multiply the DFT-order coefficients by (-1)^{j_1 + ... + j_d}, the
// factor exp(-i pi j.k_0 / L) of the grid's first point k_0 = (-L, ..., -L)
// (the parity of the signed mode j equals that of its position, N even).
template <typename T>
__global__ void k_alternate_sign(cx<T> *__restrict__ g, int d, int N, size_t nd) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nd; i += (size_t)gridDim.x * blockDim.x) {
        size_t r = i;
        int par = 0;
        for (int a = 0; a < d; ++a) {
            par += (int)(r % (size_t)N);
            r /= (size_t)N;
        }
        if (par & 1) g[i] = mkc<T>(-g[i].x, -g[i].y);
    }
}

// ------------------------------------------------------------------ pass 1
// Global field indices (fa, fb) of unit u of the chunk starting at group g0
// with ng groups; fb = -1 for a lone field.  In the shared-field layout
// (sf0 >= 0) the chunk's fields are sf0 .. sf0 + sK - 1 and unit u packs
// fields 2u and 2u + 1.
__device__ __forceinline__ void unit_fields(int u, int g0, int ng, int FPG, int PPG, const int *__restrict__ prod_local,
                                            int sf0, int sK, int &fa, int &fb) {
    if (sf0 >= 0) {
        fa = sf0 + 2 * u;
        fb = 2 * u + 1 < sK ? fa + 1 : -1;
        return;
    }
    const int ncu = (ng + 1) >> 1;
    if (u < ncu) {
        const int ga = g0 + 2 * u;
        fa = ga * FPG;
        fb = 2 * u + 1 < ng ? (ga + 1) * FPG : -1;
    } else {
        const int k = u - ncu;
        const int gl = k / PPG, p = k - gl * PPG;
        const int slot = (g0 + gl) * PPG + p;
        fa = (g0 + gl) * FPG + prod_local[2 * slot];
        fb = (g0 + gl) * FPG + prod_local[2 * slot + 1];
    }
}

// ghat(j) (E_a(j) + i E_b(j)) for one point, with E_x = row factor * tab[j]:
// the packed spectrum of the unit (fields a and b real up to their Nyquist
// parts, see pass 2).
template <typename T>
__device__ __forceinline__ cx<T> packed(cx<T> g, cx<T> ea, cx<T> eb) {
    const cx<T> e = mkc<T>(ea.x - eb.y, ea.y + eb.x);
    return cmul<T>(g, e);
}

// 3D: block (j1, unit block).  For each unit of the block: row lines take the
// packed spectrum of plane j1 and transform along axis 2 (one warp per LPW
// rows); the rows go through shared memory; then every column z is
// transformed along axis 1 by N/8 threads spread over the block, with 32
// consecutive columns per warp, so the stores to H[unit][j1][y][z] are whole
// rows.  The axis-1 and axis-2 phase rows of a unit's two fields are copied
// to shared memory (cp.async) one unit ahead of their use.
template <typename T, int N>
__global__ void __launch_bounds__(N * LineCfg<T, N>::TPL)
k_pass1_3d(const cx<T> *__restrict__ ghat, const cx<T> *__restrict__ phase, cx<T> *__restrict__ H,
           const cx<T> *__restrict__ tw_g, const int *__restrict__ prod_local, int g0, int ng, int FPG, int PPG,
           int nunits, int units_per_block, int sf0, int sK) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, WP = Work<N>::PITCH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *work = tw + N;
    cx<T> *scratch = work + N * WP;           // row scratch, then column scratch
    // 2 buffers of 4N + 2 entries: (field a, field b) x rows 1, 2, then the two
    // fields' row-0 entries at j1
    cx<T> *prow = scratch + N * LinePad<N>::PITCH;
    constexpr int PS = 4 * N + 2;
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int row = warp * LPW + c;           // axis-1 index j2 of this row line
    const int z = threadIdx.x % N, ty = threadIdx.x / N;   // column lines
    cx<T> *rscr = scratch + (size_t)row * LinePad<N>::PITCH;
    const int ubeg = blockIdx.y * units_per_block;
    const int uend = min(nunits, ubeg + units_per_block);
    const size_t NN = (size_t)N * N;
    const int j1 = blockIdx.x;
    // rows 1 and 2 of unit u's phase tables: prow[buf][0, 2N) field a, [2N, 4N)
    // field b; [4N], [4N + 1] the row-0 entries at j1 of fields a and b
    auto stage_rows = [&](int u) {
        int fa, fb;
        unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
        const cx<T> *pa = phase + (size_t)fa * 3 * N + N;
        const cx<T> *pb = phase + (size_t)(fb >= 0 ? fb : fa) * 3 * N + N;
        cx<T> *dst = prow + ((u - ubeg) & 1) * PS;
        for (int i = threadIdx.x; i < PS; i += blockDim.x)
            cp_async_cx<T>(dst + i, i < 2 * N   ? pa + i
                                    : i < 4 * N ? pb + (i - 2 * N)
                                    : (i == 4 * N ? pa : pb) - N + j1);
        cp_async_commit();
    };
    if (ubeg < uend) stage_rows(ubeg);
    const cx<T> *grow = ghat + ((size_t)j1 * N + row) * N;
    cx<T> g[E];
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = grow[t + e * TPL];
    twiddle_store<T, N>(tw, twv, tw_g);
    for (int u = ubeg; u < uend; ++u) {
        int fa, fb;
        unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
        if (u + 1 < uend) stage_rows(u + 1);   // into the buffer unit u - 1 used
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();                       // unit u's rows, copied by the whole block
        const cx<T> *ra = prow + ((u - ubeg) & 1) * PS, *rb = ra + 2 * N;
        const cx<T> a01 = cmul<T>(ra[4 * N], ra[row]);
        cx<T> v[E];
        if (fb >= 0) {
            const cx<T> b01 = cmul<T>(ra[4 * N + 1], rb[row]);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j3 = t + e * TPL;
                v[e] = packed<T>(g[e], cmul<T>(ra[N + j3], a01), cmul<T>(rb[N + j3], b01));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cmul<T>(g[e], cmul<T>(ra[N + t + e * TPL], a01));
        }
        line_fft<T, N, E, +1>(v, t, rscr, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) work[row * WP + t + e * TPL] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = work[(ty + e * TPL) * WP + z];
        col_fft<T, N, E, +1>(v, ty, scratch, z, N, tw);
        cx<T> *out = H + ((size_t)u * N + j1) * NN;
#pragma unroll
        for (int e = 0; e < E; ++e) out[(ty + e * TPL) * N + z] = v[e];
        __syncthreads();
    }
}

// Separable trailing-axis pass (3D; HostPlan::separable).  Block (j1, row
// value vi of the chunk): the rows of plane j1 of ghat times E2(j3, x2) of
// the row value are transformed along axis 2 once (warp lines, into `work`),
// then for every pair (x1, x2) of that row value the columns of the result
// times E1(j2, x1) are transformed along axis 1 (column lines, 32
// consecutive columns per warp) into the pair's plane S[pair][j1][.][.].
// The axis-0 phase E0(j1, x0) of each field is applied by the axis-0 pass.
// sep_v[3 v] = field of row value v (its axis-2 phase row), [3 v + 1],
// [3 v + 2] = first and end pair (chunk-local); sep_p[p] = field of pair p
// (its axis-1 phase row); v0 / p0 = the chunk's first row value / pair.
template <typename T, int N>
__global__ void __launch_bounds__(N * LineCfg<T, N>::TPL)
k_sep_planes_3d(const cx<T> *__restrict__ ghat, const cx<T> *__restrict__ phase, cx<T> *__restrict__ S,
                const cx<T> *__restrict__ tw_g, const int *__restrict__ sep_v, const int *__restrict__ sep_p, int v0,
                int p0) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, WP = Work<N>::PITCH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *work = tw + N;
    cx<T> *scratch = work + N * WP;           // row scratch, then column scratch
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int row = warp * LPW + c;           // j2 of this row line
    const int z = threadIdx.x % N, ty = threadIdx.x / N;   // column lines
    const int j1 = blockIdx.x, v = v0 + blockIdx.y;
    const int vf = sep_v[3 * v], pb = sep_v[3 * v + 1], pe = sep_v[3 * v + 2];
    const cx<T> *grow = ghat + ((size_t)j1 * N + row) * N;
    const cx<T> *e2 = phase + (size_t)vf * 3 * N + 2 * N;
    cx<T> x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = cmul<T>(grow[t + e * TPL], e2[t + e * TPL]);
    twiddle_store<T, N>(tw, twv, tw_g);
    line_fft<T, N, E, +1>(x, t, scratch + (size_t)row * LinePad<N>::PITCH, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) work[row * WP + t + e * TPL] = x[e];
    __syncthreads();
    const size_t NN = (size_t)N * N;
    for (int p = pb; p < pe; ++p) {
        const cx<T> *e1 = phase + (size_t)sep_p[p0 + p] * 3 * N + N;
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = cmul<T>(work[(ty + e * TPL) * WP + z], e1[ty + e * TPL]);
        col_fft<T, N, E, +1>(x, ty, scratch, z, N, tw);
        cx<T> *out = S + ((size_t)p * N + j1) * NN;
#pragma unroll
        for (int e = 0; e < E; ++e) out[(ty + e * TPL) * N + z] = x[e];
    }
}

// The same pass for N = 64 in FP32 with warp-local lines only.  Block (j1,
// row value), 512 threads: each of the 16 warps transforms 4 rows of the
// plane (lane = row + 4 t holding j3 = t + 8 e) with line64_swz in its own
// 256-entry slot and writes them to `work`; after one barrier it transforms
// 4 consecutive columns (lane = column + 4 t holding j2 = t + 8 e) for every
// pair of the row value and stores them.  The plane of ghat and the phase
// rows (E2 of the row value, E1 of each of its at most max_value_pairs
// pairs) are first copied into shared memory with cp.async.  Its planes are column-blocked:
// point (i2, i3) of a plane at sep_col64(i2 * 64 + i3), blocks of 4 columns
// one after the other, each 64 rows of 4 points: every store instruction
// writes 256 contiguous bytes.
__host__ __device__ __forceinline__ int sep_col64(int col) {
    return ((col & 63) >> 2) * 256 + (col >> 6) * 4 + (col & 3);
}

template <int N> struct SepWork64 {
    static constexpr int WP = N + 4;   // row pitch of `work` (= 4 mod 16: conflict-free column reads per half-warp)
};

template <int N>
__global__ void __launch_bounds__(512, 2)
k_sep_planes64(const float2 *__restrict__ ghat, const float2 *__restrict__ phase, float2 *__restrict__ S,
               const float2 *__restrict__ tw_g, const int *__restrict__ sep_v, const int *__restrict__ sep_p, int v0,
               int p0, int n_fields, int max_pairs, int max_value_pairs) {
    static_assert(N == 64, "64-point lines");
    constexpr int WP = SepWork64<N>::WP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tws = reinterpret_cast<float2 *>(smem_raw);            // 64 twiddles
    float2 *work = tws + N;                                          // N rows of WP
    float2 *slots = work + N * WP;                                   // 16 warps x 256
    float2 *eph = slots + 16 * 256;                                  // E2 row, then E1 rows of the pairs
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = lane & 3, t = lane >> 2;
    const int j1 = blockIdx.x, v = v0 + blockIdx.y;
    const int vf = sep_v[3 * v], pb = sep_v[3 * v + 1], pe = sep_v[3 * v + 2];
    if (!WKE_GUARD(vf >= 0 && vf < n_fields && pb >= 0 && pb <= pe && pe <= max_pairs && pe - pb <= max_value_pairs,
                   kChkSepPair))
        return;
    float2 *slot = slots + (size_t)warp * 256;
    {
        // 16-byte pieces: plane j1 of ghat (64 rows of 32, rows padded to WP in
        // `work`), then the phase rows (32 pieces each)
        const int npl = N * N / 2, nph = 32 * (1 + pe - pb);
        for (int i = tid; i < npl + nph; i += 512) {
            if (i < npl) {
                const int r = i >> 5, q = i & 31;
                cp_async16(work + r * WP + 2 * q, ghat + ((size_t)j1 * N + r) * N + 2 * q);
            } else {
                const int k = (i - npl) >> 5, q = (i - npl) & 31;
                const int f = k == 0 ? vf : sep_p[p0 + pb + k - 1];
                if (!WKE_GUARD(f >= 0 && f < n_fields, kChkSepPair)) continue;
                cp_async16(eph + k * N + 2 * q, phase + (size_t)f * 3 * N + (k == 0 ? 2 : 1) * N + 2 * q);
            }
        }
        cp_async_commit();
    }
    if (tid < N) tws[tid] = tw_g[tid];
    cp_async_wait<0>();
    __syncthreads();
    {
        // this warp's 4 rows, transformed in place
        const int j2 = 4 * warp + c;
        float2 x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = cmul<float>(work[j2 * WP + t + 8 * e], eph[t + 8 * e]);
        line64_swz(x, c, t, slot, tws);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 8; ++e) work[j2 * WP + t + 8 * e] = x[e];
    }
    __syncthreads();
    const size_t NN = (size_t)N * N;
    for (int p = pb; p < pe; ++p) {
        // (checked builds: the pair's field, whose phase row was staged)
        if (!WKE_GUARD(sep_p[p0 + p] >= 0 && sep_p[p0 + p] < n_fields, kChkSepPair)) continue;
        const float2 *e1 = eph + (1 + p - pb) * N;
        // column-blocked plane (sep_col64): this warp's 4 columns are one
        // contiguous 64 x 4 block, so each store instruction writes 256 bytes
        float2 *out = S + ((size_t)p * N + j1) * NN + (size_t)warp * 4 * N;
        {
            const int i3 = 4 * warp + c;
            float2 x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = cmul<float>(work[(t + 8 * e) * WP + i3], e1[t + 8 * e]);
            line64_swz(x, c, t, slot, tws);
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 8; ++e) out[(t + 8 * e) * 4 + c] = x[e];
        }
    }
}

// 2D: block (row block, unit).  Row j1 of the packed spectrum, inverse
// transform along axis 1 -> H[unit][j1][y].
template <typename T, int N>
__global__ void k_pass1_2d(const cx<T> *__restrict__ ghat, const cx<T> *__restrict__ phase, cx<T> *__restrict__ H,
                           const cx<T> *__restrict__ tw_g, const int *__restrict__ prod_local, int g0, int ng,
                           int FPG, int PPG, int sf0, int sK) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;
    load_twiddles<T, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    const int j1 = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    const int u = blockIdx.y;
    cx<T> *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    int fa, fb;
    unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
    const cx<T> *pa = phase + (size_t)fa * 2 * N;
    const cx<T> a0 = pa[j1];
    cx<T> v[E];
    if (fb >= 0) {
        const cx<T> *pb = phase + (size_t)fb * 2 * N;
        const cx<T> b0 = pb[j1];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j2 = t + e * TPL;
            v[e] = packed<T>(ghat[(size_t)j1 * N + j2], cmul<T>(pa[N + j2], a0), cmul<T>(pb[N + j2], b0));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
            v[e] = cmul<T>(ghat[(size_t)j1 * N + t + e * TPL], cmul<T>(pa[N + t + e * TPL], a0));
    }
    line_fft<T, N, E, +1>(v, t, scr, tw);
    cx<T> *out = H + ((size_t)u * N + j1) * N;
#pragma unroll
    for (int e = 0; e < E; ++e) out[t + e * TPL] = v[e];
}

// ------------------------------------------------------------------ Nyquist tables
// For field x and axis ax, the modes with j_ax = -N/2 (position N/2) and,
// to make the sets disjoint, no earlier axis at -N/2, give the part of
// f_N(k - x) that is not real:
//   sum_ax (-1)^{i_ax} c_ax T_ax(other indices),  c_ax = exp(i pi (N/2) x_ax / L),
// with T_ax the inverse transform over the other axes of that masked slice of
// ghat times the other axes' phases.  The table stores V_ax = Im(c_ax T_ax).
// Both kernels read the compact masked slices written by the forward pass.
// 3D: block (axis, block of units).  The two fields of a unit share one
// transform: with D_x the masked Nyquist slice times field x's phases (and
// c_ax), Im(IDFT(D_x)) = IDFT((D_x(j) - conj D_x(-j)) / (2i)), whose input is
// Hermitian, so IDFT(Dh_a + i Dh_b) = V_a + i V_b.  The unit's tables are
// stored interleaved (V_a, V_b), the layout pass 2 reads.
template <typename T>
__device__ __forceinline__ cx<T> herm_half(cx<T> d, cx<T> dm) {
    // (d - conj(dm)) / (2i)
    return mkc<T>((T)0.5 * (d.y + dm.y), (T)-0.5 * (d.x - dm.x));
}

// Grid (axis, unit of the chunk, chunk - chunk0): chunk c covers groups
// [c G, min((c + 1) G, n_groups)) and its units start at
// V + (c - chunk0) * units_per_chunk * 3 * N^2.
template <typename T, int N>
__global__ void __launch_bounds__(N * LineCfg<T, N>::TPL)
k_nyquist_3d(const cx<T> *__restrict__ phase, cx<T> *__restrict__ V, const cx<T> *__restrict__ tw_g,
             const cx<T> *__restrict__ nslice, const int *__restrict__ prod_local, int G, int n_groups, int FPG,
             int PPG, int units_per_chunk, int chunk0, int sf0, int sK) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, WP = Work<N>::PITCH, H2 = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *work = tw + N;
    cx<T> *scratch = work + N * WP;
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int row = warp * LPW + c;           // index along b0
    const int z = threadIdx.x % N, ty = threadIdx.x / N;
    cx<T> *rscr = scratch + (size_t)row * LinePad<N>::PITCH;
    const size_t NN = (size_t)N * N;
    const int ax = blockIdx.x, u = blockIdx.y;
    const int g0 = (chunk0 + blockIdx.z) * G, ng = min(G, n_groups - g0);
    if (u >= (sf0 >= 0 ? (sK + 1) / 2 : (ng + 1) / 2 + ng * PPG)) return;   // block-uniform
    V += (size_t)blockIdx.z * units_per_chunk * 3 * NN;
    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    const int mrow = (N - row) % N;
    const cx<T> *S = nslice + (size_t)ax * NN;
    int fa, fb;
    unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
    const cx<T> *pa = phase + (size_t)fa * 3 * N;
    const cx<T> ca = pa[ax * N + H2];
    const cx<T> ra = cmul<T>(ca, pa[b0 * N + row]), rma = cmul<T>(ca, pa[b0 * N + mrow]);
    const cx<T> *pb = fb >= 0 ? phase + (size_t)fb * 3 * N : pa;
    const cx<T> cb = pb[ax * N + H2];
    const cx<T> rb = cmul<T>(cb, pb[b0 * N + row]), rmb = cmul<T>(cb, pb[b0 * N + mrow]);
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int col = t + e * TPL, mcol = (N - col) % N;
        const cx<T> s0 = S[(size_t)row * N + col], s1 = S[(size_t)mrow * N + mcol];
        const cx<T> ha = herm_half<T>(cmul<T>(s0, cmul<T>(ra, pa[b1 * N + col])),
                                      cmul<T>(s1, cmul<T>(rma, pa[b1 * N + mcol])));
        cx<T> hb = mkc<T>((T)0, (T)0);
        if (fb >= 0)
            hb = herm_half<T>(cmul<T>(s0, cmul<T>(rb, pb[b1 * N + col])), cmul<T>(s1, cmul<T>(rmb, pb[b1 * N + mcol])));
        v[e] = mkc<T>(ha.x - hb.y, ha.y + hb.x);
    }
    twiddle_store<T, N>(tw, twv, tw_g);
    line_fft<T, N, E, +1>(v, t, rscr, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) work[row * WP + t + e * TPL] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = work[(ty + e * TPL) * WP + z];
    col_fft<T, N, E, +1>(v, ty, scratch, z, N, tw);
    cx<T> *out = V + ((size_t)u * 3 + ax) * NN;
#pragma unroll
    for (int e = 0; e < E; ++e) out[(ty + e * TPL) * N + z] = v[e];
}

// The same tables for N = 64 in FP32 with warp-local lines (the layout of
// k_sep_planes64): block (axis, unit), 512 threads.  The block first copies
// the axis's Nyquist slice (64 x 64, rows padded to WP) and the two fields'
// phase rows into shared memory with cp.async; then warp w forms the input of
// rows 4 w .. 4 w + 3 (lane = row + 4 t holding columns t + 8 e), transforms
// them with line64_swz in its own slot and writes them to `work`; after one
// barrier it transforms columns 4 w .. 4 w + 3 and stores the table.
template <int N>
__global__ void __launch_bounds__(512, 1)
k_nyquist64(const float2 *__restrict__ phase, float2 *__restrict__ V, const float2 *__restrict__ tw_g,
            const float2 *__restrict__ nslice, const int *__restrict__ prod_local, int G, int n_groups, int FPG,
            int PPG, int units_per_chunk, int chunk0, int sf0, int sK) {
    static_assert(N == 64, "64-point lines");
    constexpr int WP = SepWork64<N>::WP, H2 = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tws = reinterpret_cast<float2 *>(smem_raw);            // 64 twiddles
    float2 *work = tws + N;                                          // N rows of WP
    float2 *slots = work + N * WP;                                   // 16 warps x 256
    float2 *sl = slots + 16 * 256;                                   // the slice: N rows of WP
    float2 *ph = sl + N * WP;                                        // phase rows: field a (3 N), field b (3 N)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = lane & 3, t = lane >> 2;
    float2 *slot = slots + (size_t)warp * 256;
    const size_t NN = (size_t)N * N;
    const int ax = blockIdx.x, u = blockIdx.y;
    const int g0 = (chunk0 + blockIdx.z) * G, ng = min(G, n_groups - g0);
    if (u >= (sf0 >= 0 ? (sK + 1) / 2 : (ng + 1) / 2 + ng * PPG)) return;   // block-uniform
    V += (size_t)blockIdx.z * units_per_chunk * 3 * NN;
    int fa, fb;
    unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
    {
        // 16-byte pieces: the slice's 64 rows of 32 pieces, then 2 x 96 phase pieces
        const float2 *S = nslice + (size_t)ax * NN;
        for (int i = tid; i < N * N / 2; i += 512) {
            const int r = i >> 5, q = i & 31;
            cp_async16(sl + r * WP + 2 * q, S + (size_t)r * N + 2 * q);
        }
        if (tid < 3 * N) {
            const int f = tid < 3 * N / 2 ? fa : (fb >= 0 ? fb : fa), q = tid % (3 * N / 2);
            cp_async16(ph + (tid < 3 * N / 2 ? 0 : 3 * N) + 2 * q, phase + (size_t)f * 3 * N + 2 * q);
        }
        cp_async_commit();
    }
    if (tid < N) tws[tid] = tw_g[tid];
    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    const float2 *pa = ph, *pb = ph + 3 * N;
    cp_async_wait<0>();
    __syncthreads();
    {
        const int row = 4 * warp + c, mrow = (N - row) % N;
        const float2 ca = pa[ax * N + H2], cb = pb[ax * N + H2];
        const float2 ra = cmul<float>(ca, pa[b0 * N + row]), rma = cmul<float>(ca, pa[b0 * N + mrow]);
        const float2 rb = cmul<float>(cb, pb[b0 * N + row]), rmb = cmul<float>(cb, pb[b0 * N + mrow]);
        float2 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int col = t + 8 * e, mcol = (N - col) % N;
            const float2 s0 = sl[row * WP + col], s1 = sl[mrow * WP + mcol];
            const float2 ha = herm_half<float>(cmul<float>(s0, cmul<float>(ra, pa[b1 * N + col])),
                                               cmul<float>(s1, cmul<float>(rma, pa[b1 * N + mcol])));
            float2 hb = make_float2(0.f, 0.f);
            if (fb >= 0)
                hb = herm_half<float>(cmul<float>(s0, cmul<float>(rb, pb[b1 * N + col])),
                                      cmul<float>(s1, cmul<float>(rmb, pb[b1 * N + mcol])));
            v[e] = make_float2(ha.x - hb.y, ha.y + hb.x);
        }
        line64_swz(v, c, t, slot, tws);
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 8; ++e) work[row * WP + t + 8 * e] = v[e];
    }
    __syncthreads();
    {
        const int z = 4 * warp + c;
        float2 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = work[(t + 8 * e) * WP + z];
        line64_swz(v, c, t, slot, tws);
        float2 *out = V + ((size_t)u * 3 + ax) * NN;
#pragma unroll
        for (int e = 0; e < 8; ++e) out[(size_t)(t + 8 * e) * N + z] = v[e];
    }
}

// 2D: item = (unit, axis); the slice is a line along the other axis.  One
// warp per block holds LPW items (one line each).
template <typename T, int N>
__global__ void __launch_bounds__(32)
k_nyquist_2d(const cx<T> *__restrict__ phase, cx<T> *__restrict__ V, const cx<T> *__restrict__ tw_g,
             const cx<T> *__restrict__ nslice, const int *__restrict__ prod_local, int G, int n_groups, int FPG,
             int PPG, int units_per_chunk, int chunk0, int sf0, int sK) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, H2 = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;
    load_twiddles<T, N>(tw, tw_g);
    const int lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int g0 = (chunk0 + blockIdx.y) * G, ng = min(G, n_groups - g0);
    const int nitems = 2 * (sf0 >= 0 ? (sK + 1) / 2 : (ng + 1) / 2 + ng * PPG);
    V += (size_t)blockIdx.y * units_per_chunk * 2 * N;
    const int item = blockIdx.x * LPW + c;
    const bool valid = item < nitems;
    const int it = valid ? item : nitems - 1;
    const int u = it >> 1, ax = it & 1;
    const int b = 1 - ax;
    int fa, fb;
    unit_fields(u, g0, ng, FPG, PPG, prod_local, sf0, sK, fa, fb);
    const cx<T> *pa = phase + (size_t)fa * 2 * N;
    const cx<T> *pb = fb >= 0 ? phase + (size_t)fb * 2 * N : pa;
    const cx<T> ca = pa[ax * N + H2], cb = pb[ax * N + H2];
    const cx<T> *S = nslice + (size_t)ax * N;
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int jb = t + e * TPL, mj = (N - jb) % N;
        const cx<T> s0 = S[jb], s1 = S[mj];
        const cx<T> ha = herm_half<T>(cmul<T>(s0, cmul<T>(ca, pa[b * N + jb])), cmul<T>(s1, cmul<T>(ca, pa[b * N + mj])));
        cx<T> hb = mkc<T>((T)0, (T)0);
        if (fb >= 0)
            hb = herm_half<T>(cmul<T>(s0, cmul<T>(cb, pb[b * N + jb])), cmul<T>(s1, cmul<T>(cb, pb[b * N + mj])));
        v[e] = mkc<T>(ha.x - hb.y, ha.y + hb.x);
    }
    line_fft<T, N, E, +1>(v, t, scratch + (size_t)c * LinePad<N>::PITCH, tw);
    if (valid) {
        cx<T> *out = V + ((size_t)u * 2 + ax) * N;
#pragma unroll
        for (int e = 0; e < E; ++e) out[t + e * TPL] = v[e];
    }
}

// ------------------------------------------------------------------ pass 2
// Block (column tile, group of the chunk).  A tile is CB consecutive columns
// of the trailing axes; each column's N points along axis 0 are held by
// TPL = N/E threads spread over the block (thread ty holds points
// ty + e TPL), so every warp reads and writes 32 consecutive columns of one
// row.  The block transforms C once and keeps s = C + F and cf = C F; for
// every product of the group it transforms the unit holding A and B (two
// fields packed in one transform) and adds (A B) s - cf (A + B).  The
// group's sum goes to that group's double accumulator.
// Points per thread EP: 4 (radices 4, 4, 4 for N = 64; fewer registers, more
// blocks per SM) or 8 (radices 8, 8; fewer instructions).  The plan's tuning
// picks one; N >= 128 always uses 8, and lengths 3 * 2^a use 12 (radices 12
// then powers of two).
template <typename T, int N, int EP> struct Pass2Cfg {
    static constexpr int E = N % 3 == 0 ? 12 : N >= 128 ? 8 : EP;
    static constexpr int TPL = N / E;                    // threads per column
    // 128 threads for 12 double points per thread, so that the two staged
    // tiles and the scratch fit in shared memory
    static constexpr int THREADS = (E == 12 && sizeof(T) == 8) ? 128 : 256;
    static constexpr int CB = THREADS / TPL;             // columns per block (at most)
    static constexpr int MIN_BLOCKS = E == 12 ? 1 : sizeof(T) == 4 ? (E == 4 ? 3 : 2) : (E == 4 ? 2 : 1);
    static_assert(THREADS % TPL == 0 && TPL % 2 == 0, "threads per column must divide the block and be even");
};

// Imaginary parts of the Nyquist contributions of a unit's two fields at
// point (i1, column): sum_ax (-1)^{i_ax} V_ax(other indices), real-slot field
// in .x and imaginary-slot field in .y.  `Vu` holds the unit's d interleaved
// tables; the column is (i2, i3) in 3D, i2 in 2D; sgn1 = (-1)^{i1}.
template <typename T, int N>
__device__ __forceinline__ cx<T> nyq_pair(const cx<T> *__restrict__ Vu, int d, int i1, int col, T sgn1) {
    if (d == 3) {
        const int i2 = col / N, i3 = col - i2 * N;
        const T sg2 = (i2 & 1) ? (T)-1 : (T)1, sg3 = (i3 & 1) ? (T)-1 : (T)1;
        const cx<T> v0 = Vu[col];
        const cx<T> v1 = Vu[N * N + i1 * N + i3];
        const cx<T> v2 = Vu[2 * N * N + i1 * N + i2];
        return mkc<T>(sgn1 * v0.x + sg2 * v1.x + sg3 * v2.x, sgn1 * v0.y + sg2 * v1.y + sg3 * v2.y);
    }
    const T sg2 = (col & 1) ? (T)-1 : (T)1;
    const cx<T> v0 = Vu[col];
    const cx<T> v1 = Vu[N + i1];
    return mkc<T>(sgn1 * v0.x + sg2 * v1.x, sgn1 * v0.y + sg2 * v1.y);
}

// Block (column tile, group of the chunk).  The group's C unit holds C in its
// real slot (even group of a pair) or imaginary slot (odd group); each
// product unit holds A (real slot) and B (imaginary slot).  With the unit's
// axis-0 transform Z and the Nyquist imaginary parts a (of the real-slot
// field) and b (of the imaginary-slot field):
//   real-slot field = (Re Z + b) + i a,  imaginary-slot field = (Im Z - a) + i b.
// Then, keeping s = C + F and cf = C F, each product contributes
// A B (C + F) - C F (A + B) = (A B) s - cf (A + B), written out in real parts.
template <typename T, int N, int EP, bool IM, bool NYQ>
__global__ void __launch_bounds__(Pass2Cfg<T, N, EP>::THREADS, Pass2Cfg<T, N, EP>::MIN_BLOCKS)
k_pass2(const cx<T> *__restrict__ H, const cx<T> *__restrict__ Vtab, const T *__restrict__ f,
        double *__restrict__ Qacc, double *__restrict__ Qim, const int *__restrict__ prod_local,
        const double *__restrict__ prod_W, const cx<T> *__restrict__ tw_g, int d, int P, int CB, int PPG, int g0,
        int ng) {
    typedef Pass2Cfg<T, N, EP> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;                  // LinePad<N>::LEN rows x CB columns
    cx<T> *stage = scratch + LinePad<N>::LEN * CB;   // 2 tiles of N x CB, prefetched
    // 3D with the Nyquist set kept and a tile inside one row of the trailing
    // axes: each unit's table entries for the tile are staged with it in one
    // of 3 slots (a slot is rewritten only after a full transform, with its
    // barriers, since its last read): V_1(i1, i3) for the tile's columns (each
    // thread copies what it reads), V_2(i1, i2) of the tile's row (copied by
    // the threads of column 0) and V_0 of the tile's columns.
    const bool vstage = NYQ && d == 3 && (N % CB) == 0;
    const int VSLOT = N * CB + N + CB;
    cx<T> *vbuf = stage + 2 * N * CB;
    load_twiddles<T, N>(tw, tw_g);
    const int z = threadIdx.x % CB, t = threadIdx.x / CB;
    const int col = blockIdx.x * CB + z;
    const int i2 = col / N, i3 = col - i2 * N;
    const int gl = blockIdx.y;
    const size_t ND = (size_t)N * P;
    const size_t VS = (size_t)d * (ND / N);   // Nyquist table entries per unit
    const int ncu = (ng + 1) >> 1;
    const cx<T> *Hc = H + (size_t)(gl >> 1) * ND;                       // this group's C unit
    const cx<T> *Hp = H + (size_t)(ncu + gl * PPG) * ND;               // its product units
    const cx<T> *Vc = Vtab + (size_t)(gl >> 1) * VS;
    const cx<T> *Vp = Vtab + (size_t)(ncu + gl * PPG) * VS;
    const T sgn1 = (t & 1) ? (T)-1 : (T)1;    // (-1)^{i1}: TPL is even, so i1 = t + e TPL has t's parity
    const T sg2 = (i2 & 1) ? (T)-1 : (T)1, sg3 = (i3 & 1) ? (T)-1 : (T)1;
    const int tiles = 1 + PPG;
    auto prefetch = [&](int k) {
        const cx<T> *src = k == 0 ? Hc : Hp + (size_t)(k - 1) * ND;
        cx<T> *dst = stage + (k & 1) * N * CB;
#pragma unroll
        for (int e = 0; e < E; ++e)
            cp_async_cx<T>(dst + (t + e * TPL) * CB + z, src + (size_t)(t + e * TPL) * P + col);
        if (vstage) {
            const cx<T> *vs = k == 0 ? Vc : Vp + (size_t)(k - 1) * VS;
            cx<T> *vd = vbuf + (k % 3) * VSLOT;
#pragma unroll
            for (int e = 0; e < E; ++e)
                cp_async_cx<T>(vd + (t + e * TPL) * CB + z, vs + N * N + (t + e * TPL) * N + i3);
            if (z == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) cp_async_cx<T>(vd + N * CB + t + e * TPL, vs + 2 * N * N + (t + e * TPL) * N + i2);
            }
            if (t == 0) cp_async_cx<T>(vd + N * CB + N + z, vs + col);
        }
        cp_async_commit();
    };
    // Nyquist imaginary parts of tile k's unit at (i1, this column) from the
    // staged slot (same sum as nyq_pair)
    auto nyq_staged = [&](int k, int i1) -> cx<T> {
        const cx<T> *vd = vbuf + (k % 3) * VSLOT;
        const cx<T> v0 = vd[N * CB + N + z], v1 = vd[i1 * CB + z], v2 = vd[N * CB + i1];
        return mkc<T>(sgn1 * v0.x + sg2 * v1.x + sg3 * v2.x, sgn1 * v0.y + sg2 * v1.y + sg3 * v2.y);
    };
    auto take = [&](int k, cx<T> (&v)[E]) {
        const cx<T> *src = stage + (k & 1) * N * CB;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = src[(t + e * TPL) * CB + z];
    };

    prefetch(0);
    if (tiles > 1) prefetch(1);
    else cp_async_commit();
    cx<T> v[E];
    T sr[E], si[E], cr[E], ci[E];
    cp_async_wait<1>();
    take(0, v);
    col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);   // its barriers also order the stage reads
    {
        const bool odd = gl & 1;
        const bool has_partner = (gl ^ 1) < ng;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i1 = t + e * TPL;
            T re = odd ? v[e].y : v[e].x, im = (T)0;
            if (NYQ) {
                const cx<T> ab = vstage ? nyq_staged(0, i1) : nyq_pair<T, N>(Vc, d, i1, col, sgn1);
                const T self = odd ? ab.y : ab.x, part = has_partner ? (odd ? ab.x : ab.y) : (T)0;
                re += odd ? -part : part;
                im = self;
            }
            const T F = f[(size_t)i1 * P + col];
            sr[e] = re + F;
            si[e] = im;
            cr[e] = re * F;
            ci[e] = im * F;
        }
    }
    T ar[E], ai[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        ar[e] = (T)0;
        ai[e] = (T)0;
    }
    const double *Wg = prod_W + (size_t)(g0 + gl) * PPG;
    for (int p = 0; p < PPG; ++p) {
        const T W = (T)Wg[p];
        if (p + 2 < tiles) prefetch(p + 2);   // buffer of tile p, already read
        else cp_async_commit();               // empty group keeps the count uniform
        cp_async_wait<1>();
        take(p + 1, v);
        col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i1 = t + e * TPL;
            T a = (T)0, b = (T)0;
            if (NYQ) {
                const cx<T> ab = vstage ? nyq_staged(p + 1, i1) : nyq_pair<T, N>(Vp + (size_t)p * VS, d, i1, col, sgn1);
                a = ab.x;
                b = ab.y;
            }
            const T Ar = v[e].x + b, Br = v[e].y - a;          // A = Ar + i a, B = Br + i b
            const T pr = Ar * Br - a * b, pim = Ar * b + a * Br;   // A B
            const T ur = Ar + Br, ui = a + b;                  // A + B
            ar[e] += W * ((pr * sr[e] - pim * si[e]) - (cr[e] * ur - ci[e] * ui));
            if (IM) ai[e] += W * ((pr * si[e] + pim * sr[e]) - (cr[e] * ui + ci[e] * ur));
        }
    }
    cp_async_wait<0>();
    double *Qg = Qacc + (size_t)gl * ND;
#pragma unroll
    for (int e = 0; e < E; ++e) Qg[(size_t)(t + e * TPL) * P + col] += (double)ar[e];
    if (IM) {
        double *Qig = Qim + (size_t)gl * ND;
#pragma unroll
        for (int e = 0; e < E; ++e) Qig[(size_t)(t + e * TPL) * P + col] += (double)ai[e];
    }
}

// ------------------------------------------------------------------ shared-field layout
// Pass 2: axis-0 inverse transform of every unit of the chunk, in place.
// Block (column tile, unit); the tile layout of pass 2.
template <typename T, int N, int EP>
__global__ void __launch_bounds__(Pass2Cfg<T, N, EP>::THREADS)
k_axis0(cx<T> *__restrict__ H, const cx<T> *__restrict__ tw_g, int P, int CB) {
    typedef Pass2Cfg<T, N, EP> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;                  // LinePad<N>::LEN rows x CB columns
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int z = threadIdx.x % CB, t = threadIdx.x / CB;
    const int col = blockIdx.x * CB + z;
    cx<T> *Hu = H + (size_t)blockIdx.y * N * P + col;
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = Hu[(size_t)(t + e * TPL) * P];
    twiddle_store<T, N>(tw, twv, tw_g);
    col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) Hu[(size_t)(t + e * TPL) * P] = v[e];
}

// Separable plans: the axis-0 input of unit u (fields a, b) from the pair
// planes, E0(j1, x0a) S_a(j1, col) + i E0(j1, x0b) S_b(j1, col), the packed
// spectrum's transform over the trailing axes (exact: the phases factor per
// axis).  `fb` < 0 for a lone field.
template <typename T>
__device__ __forceinline__ cx<T> sep_input(const cx<T> *__restrict__ sa, const cx<T> *__restrict__ sb,
                                           const cx<T> *__restrict__ ea, const cx<T> *__restrict__ eb, int j1,
                                           size_t stride, bool pair) {
    const cx<T> A = cmul<T>(sa[(size_t)j1 * stride], ea[j1]);
    if (!pair) return A;
    const cx<T> B = cmul<T>(sb[(size_t)j1 * stride], eb[j1]);
    return mkc<T>(A.x - B.y, A.y + B.x);
}

// Axis-0 transform of every unit of a separable chunk, from the pair planes
// into H (the layout k_axis0 leaves).  Block (column tile, unit).
template <typename T, int N, int EP>
__global__ void __launch_bounds__(Pass2Cfg<T, N, EP>::THREADS)
k_axis0_sep(const cx<T> *__restrict__ S, const cx<T> *__restrict__ phase, const int *__restrict__ field_pair,
            cx<T> *__restrict__ H, const cx<T> *__restrict__ tw_g, int P, int CB, int sf0, int K, int max_pairs) {
    typedef Pass2Cfg<T, N, EP> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;                  // LinePad<N>::LEN rows x CB columns
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int z = threadIdx.x % CB, t = threadIdx.x / CB;
    const int col = blockIdx.x * CB + z;
    const int u = blockIdx.y, fa = sf0 + 2 * u;
    const bool pair = 2 * u + 1 < K;
    const int fb = pair ? fa + 1 : fa;
    const size_t ND = (size_t)N * P;
    const int qa = field_pair[fa], qb = field_pair[fb];
    if (!WKE_GUARD(qa >= 0 && qa < max_pairs && qb >= 0 && qb < max_pairs, kChkAxis0Unit)) return;
    // the FP32 N = 64 planes are column-blocked (k_sep_planes64)
    const int scol = (N == 64 && sizeof(T) == 4) ? sep_col64(col) : col;
    const cx<T> *sa = S + (size_t)qa * ND + scol, *sb = S + (size_t)qb * ND + scol;
    const cx<T> *ea = phase + (size_t)fa * 3 * N, *eb = phase + (size_t)fb * 3 * N;
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = sep_input<T>(sa, sb, ea, eb, t + e * TPL, P, pair);
    twiddle_store<T, N>(tw, twv, tw_g);
    col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
    cx<T> *Hu = H + (size_t)u * ND + col;
#pragma unroll
    for (int e = 0; e < E; ++e) Hu[(size_t)(t + e * TPL) * P] = v[e];
}

// Split-precision axis-0 transform on the tensor cores (WKE_SPLIT).  The
// inverse N-point DFT of every column of a tile of CB = 32 columns is the
// real GEMM
//   [Re Z; Im Z] = [[Re F, -Im F], [Im F, Re F]] [Re H; Im H],
//   F[i1][j1] = exp(+2 pi i i1 j1 / N)            (2N x 2N times 2N x 32),
// computed with mma.sync m16n8k8 in TF32.  Each operand x is split into
// x_hi = x rounded to TF32 and x_lo = (x - x_hi) rounded to TF32, and
// A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo is below
// 2^-22 |A| |B|), each 8-wide k-step on the tensor cores and the 2N / 8 step
// sums added in FP32.  The F entries come from the
// twiddle table.  Warp w owns output rows 16 w .. 16 w + 15 of Re Z and of
// Im Z, so each thread holds the real and imaginary parts of the same points.
// mma.sync m16n8k8 fragments (g = lane / 4, q = lane % 4): A a0 (g, q),
// a1 (g + 8, q), a2 (g, q + 4), a3 (g + 8, q + 4); B b0 (k = q, n = g),
// b1 (q + 4, g); C c0 (g, 2q), c1 (g, 2q + 1), c2 (g + 8, 2q), c3 (g + 8, 2q + 1).
__device__ __forceinline__ unsigned tf32_round(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void tf32_split(float x, unsigned &hi, unsigned &lo) {
    hi = tf32_round(x);
    lo = tf32_round(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int N>
__global__ void __launch_bounds__(N / 16 * 32)
k_axis0_tc(float2 *__restrict__ H, const float2 *__restrict__ tw_g, int P) {
    constexpr int CB = 32, K = 2 * N, LD = CB + 8;   // LD: conflict-free B fragment reads
    __shared__ float2 tw[N];
    __shared__ float Bs[K * LD];
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    float2 *Hu = H + (size_t)blockIdx.y * N * P + (size_t)blockIdx.x * CB;
    for (int i = threadIdx.x; i < N * CB; i += blockDim.x) {
        const int j1 = i / CB, c = i - j1 * CB;
        const float2 h = Hu[(size_t)j1 * P + c];
        Bs[j1 * LD + c] = h.x;
        Bs[(N + j1) * LD + c] = h.y;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[t][nt][e] = 0.0f;
    for (int kk = 0; kk < K / 8; ++kk) {
        unsigned ahi[2][4], alo[2][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i1 = 16 * warp + g + ((e & 1) ? 8 : 0);
            const int k = 8 * kk + q + ((e & 2) ? 4 : 0);
            const int half = k >= N, j1 = half ? k - N : k;
            const float2 w = tw[(i1 * j1) & (N - 1)];
            // row of Re Z: (Re F, -Im F); row of Im Z: (Im F, Re F)
            tf32_split(half ? -w.y : w.x, ahi[0][e], alo[0][e]);
            tf32_split(half ? w.x : w.y, ahi[1][e], alo[1][e]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            unsigned bhi0, blo0, bhi1, blo1;
            tf32_split(Bs[(8 * kk + q) * LD + 8 * nt + g], bhi0, blo0);
            tf32_split(Bs[(8 * kk + q + 4) * LD + 8 * nt + g], bhi1, blo1);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                // each 8-wide k-step sums into a fresh fragment, added to the
                // running sum with a rounded FP32 addition (the tensor cores'
                // own accumulation over all 2N terms loses more)
                float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                mma_tf32(part, alo[t], bhi0, bhi1);
                mma_tf32(part, ahi[t], blo0, blo1);
                mma_tf32(part, ahi[t], bhi0, bhi1);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[t][nt][e] += part[e];
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i1 = 16 * warp + g + ((e & 2) ? 8 : 0);
            const int c = 8 * nt + 2 * q + (e & 1);
            Hu[(size_t)i1 * P + c] = make_float2(acc[0][nt][e], acc[1][nt][e]);
        }
}

// Product pass: one grid point per thread and loop.  The chunk's K fields at
// the point are unpacked from the transformed units (real-slot field
// (Re Z + b) + i a, imaginary-slot field (Im Z - a) + i b, a and b the
// Nyquist imaginary parts) into this thread's column of shared memory; then
// every group g of the chunk adds, with s = C + F and cf = C F,
//   sum_p W_p Re[(A_p B_p) s - cf (A_p + B_p)]   (and Im on request).
// The chunk's product table (field slots and weights) is copied to shared
// memory once per block.  The group sums are added in T with compensation
// (Neumaier) and the chunk's total goes to the single FP64 accumulator: one
// addition per point per chunk, in chunk order, so the result is
// deterministic.
constexpr int kProductThreads = 128;
// dynamic shared memory a block may opt in to (227 KB)
constexpr size_t kMaxDynamicSmem = 227 * 1024;

// One product of the chunk's table: the two field slots (field id * blockDim,
// below 2^16) packed in one word, and the weight.
template <typename T> struct __align__(2 * sizeof(T)) ProdEntry {
    unsigned ab;
    T w;
};

template <typename T, bool IM, bool NYQ, int PPGC>
__global__ void __launch_bounds__(kProductThreads)
k_products(const cx<T> *__restrict__ H, const cx<T> *__restrict__ Vtab, const T *__restrict__ f,
           double *__restrict__ Qacc, double *__restrict__ Qim, const int *__restrict__ group_cfield,
           const int *__restrict__ prod_local, const double *__restrict__ prod_W, int d, int N, int P,
           int g0, int ng, int K, int PPG) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int stride = blockDim.x;
    cx<T> *fbase = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *fb = fbase + threadIdx.x;          // field k at fb[k * stride]
    ProdEntry<T> *ptab = reinterpret_cast<ProdEntry<T> *>(fbase + (size_t)K * stride);
    int *ctab = reinterpret_cast<int *>(ptab + ng * PPG);
    for (int i = threadIdx.x; i < ng * PPG; i += stride) {
        const int slot = g0 * PPG + i;
        ptab[i] = ProdEntry<T>{(unsigned)(prod_local[2 * slot] * stride) | ((unsigned)(prod_local[2 * slot + 1] * stride) << 16),
                               (T)prod_W[slot]};
    }
    for (int i = threadIdx.x; i < ng; i += stride) ctab[i] = group_cfield[g0 + i] * stride;
    __syncthreads();
    // N^d < 2^31 for every compiled length: point indices are 32-bit
    const unsigned ND = (unsigned)N * (unsigned)P;
    const size_t VS = (size_t)d * P;          // Nyquist table entries per unit
    const int U = (K + 1) / 2;
    const int ppg = PPGC > 0 ? PPGC : PPG;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ND; idx += gridDim.x * blockDim.x) {
        const int i1 = (int)(idx / (unsigned)P), col = (int)(idx - (unsigned)i1 * (unsigned)P);
        const T sgn1 = (i1 & 1) ? (T)-1 : (T)1;
        // offsets and signs of this point's table entries (three in 3D, two in 2D)
        int o1, o2 = 0;
        T s1, s2 = (T)0;
        if (d == 3) {
            const int i2 = (int)((unsigned)col / (unsigned)N), i3 = col - i2 * N;
            o1 = N * N + i1 * N + i3;
            o2 = 2 * N * N + i1 * N + i2;
            s1 = (i2 & 1) ? (T)-1 : (T)1;
            s2 = (i3 & 1) ? (T)-1 : (T)1;
        } else {
            o1 = N + i1;
            s1 = (col & 1) ? (T)-1 : (T)1;
        }
        const cx<T> *Hp = H + idx;
        const cx<T> *Vu = Vtab;
        for (int u = 0; u < U; ++u, Hp += ND, Vu += VS) {
            const cx<T> Z = *Hp;
            T a = (T)0, b = (T)0;
            if (NYQ) {
                const cx<T> v0 = Vu[col], v1 = Vu[o1];
                a = sgn1 * v0.x + s1 * v1.x;
                b = sgn1 * v0.y + s1 * v1.y;
                if (d == 3) {
                    const cx<T> v2 = Vu[o2];
                    a += s2 * v2.x;
                    b += s2 * v2.y;
                }
            }
            fb[(2 * u) * stride] = mkc<T>(Z.x + b, a);
            if (2 * u + 1 < K) fb[(2 * u + 1) * stride] = mkc<T>(Z.y - a, b);
        }
        const T F = f[idx];
        T sum = (T)0, comp = (T)0, sumi = (T)0, compi = (T)0;
        const ProdEntry<T> *pe = ptab;
        for (int g = 0; g < ng; ++g) {
            const cx<T> C = fb[ctab[g]];
            const T sr = C.x + F, si = C.y, cr = C.x * F, ci = C.y * F;
            T acc = (T)0, acci = (T)0;
#pragma unroll
            for (int p = 0; p < ppg; ++p, ++pe) {
                const ProdEntry<T> e = *pe;
                const cx<T> A = fb[e.ab & 0xffffu], B = fb[e.ab >> 16];
                const T pr = A.x * B.x - A.y * B.y, pim = A.x * B.y + A.y * B.x;   // A B
                const T ur = A.x + B.x, ui = A.y + B.y;                            // A + B
                acc += e.w * ((pr * sr - pim * si) - (cr * ur - ci * ui));
                if (IM) acci += e.w * ((pr * si + pim * sr) - (cr * ui + ci * ur));
            }
            // Neumaier summation of the group sums
            T tsum = sum + acc;
            comp += fabs(sum) >= fabs(acc) ? (sum - tsum) + acc : (acc - tsum) + sum;
            sum = tsum;
            if (IM) {
                tsum = sumi + acci;
                compi += fabs(sumi) >= fabs(acci) ? (sumi - tsum) + acci : (acci - tsum) + sumi;
                sumi = tsum;
            }
        }
        Qacc[idx] += (double)sum + (double)comp;
        if (IM) Qim[idx] += (double)sumi + (double)compi;
    }
}

// Product pass with staged inputs (3D, and 2D rows of at least a block).
// Block b holds the kProductThreads consecutive points p0 = b kProductThreads,
// ... of one i1 row (P is a multiple of the block).  Before any arithmetic the
// block issues, all at once with cp.async, the copies of each unit's packed
// values at its points (into field slot 2u), of the unit's V_0 entries at its
// columns (slot 2u + 1) and of the other tables' entries its points use (a
// table area of TS entries per unit: in 3D the row V_1(i1, .) and the W2
// entries V_2(i1, i2lo ..), in 2D V_1(i1)); the unit loop and the products
// then read shared memory only.  Same arithmetic, in the same order, as
// k_products.
template <typename T, bool IM, bool NYQ, int PPGC>
__global__ void __launch_bounds__(kProductThreads)
k_products_staged(const cx<T> *__restrict__ H, const cx<T> *__restrict__ Vtab, const T *__restrict__ f,
                  double *__restrict__ Qacc, double *__restrict__ Qim, const int *__restrict__ group_cfield,
                  const int *__restrict__ prod_local, const double *__restrict__ prod_W, int d, int N, int P,
                  int g0, int ng, int K, int PPG, int TS, int W2) {
    constexpr int B = kProductThreads;
    constexpr int PER16 = 16 / (int)sizeof(cx<T>);   // entries per 16-byte copy
    constexpr int PIECES = B / PER16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int U = (K + 1) / 2;
    cx<T> *fbase = reinterpret_cast<cx<T> *>(smem_raw);   // 2U slots of B points
    cx<T> *tabs = fbase + (size_t)2 * U * B;
    ProdEntry<T> *ptab = reinterpret_cast<ProdEntry<T> *>(tabs + (NYQ ? (size_t)U * TS : 0));
    int *ctab = reinterpret_cast<int *>(ptab + ng * PPG);
    const unsigned ND = (unsigned)N * (unsigned)P;
    const unsigned p0 = blockIdx.x * B;
    const int i1 = (int)(p0 / (unsigned)P), col0 = (int)(p0 - (unsigned)i1 * (unsigned)P);
    const int i2lo = col0 / N;
    const size_t VS = (size_t)d * P;          // Nyquist table entries per unit
    // each thread walks (unit u, piece k) of its copies as i = tid, tid + B, ...
    // with (u, k) = (i / R, i % R) stepped by (B / R, B % R): no division per copy
    auto walk = [](int U_, int R, auto &&copy) {
        int u = (int)threadIdx.x / R, k = (int)threadIdx.x - u * R;
        const int du = B / R, dk = B - du * R;
        while (u < U_) {
            copy(u, k);
            u += du;
            k += dk;
            if (k >= R) {
                k -= R;
                ++u;
            }
        }
    };
    {
        const cx<T> *hz = H + p0;
        const cx<T> *v0 = Vtab + col0;
        walk(U, PIECES, [&](int u, int k) {
            cp_async16(fbase + (size_t)(2 * u) * B + k * PER16, hz + (size_t)u * ND + k * PER16);
            if (NYQ) cp_async16(fbase + (size_t)(2 * u + 1) * B + k * PER16, v0 + (size_t)u * VS + k * PER16);
        });
    }
    if (NYQ && d == 3) {
        const cx<T> *v1 = Vtab + (size_t)P + (size_t)i1 * N;
        walk(U, N / PER16, [&](int u, int k) {
            cp_async16(tabs + (size_t)u * TS + k * PER16, v1 + (size_t)u * VS + k * PER16);
        });
        const cx<T> *v2 = Vtab + (size_t)2 * P + (size_t)i1 * N + i2lo;
        walk(U, min(W2, N - i2lo), [&](int u, int k) {
            cp_async_cx<T>(tabs + (size_t)u * TS + N + k, v2 + (size_t)u * VS + k);
        });
    } else if (NYQ) {
        for (int u = threadIdx.x; u < U; u += B) cp_async_cx<T>(tabs + (size_t)u * TS, Vtab + (size_t)u * VS + N + i1);
    }
    cp_async_commit();
    for (int i = threadIdx.x; i < ng * PPG; i += B) {
        const int slot = g0 * PPG + i;
        int la = prod_local[2 * slot], lb = prod_local[2 * slot + 1];
        if (!WKE_GUARD(la >= 0 && la < K && lb >= 0 && lb < K, kChkProductsSlot)) la = lb = 0;
        ptab[i] = ProdEntry<T>{(unsigned)(la * B) | ((unsigned)(lb * B) << 16), (T)prod_W[slot]};
    }
    for (int i = threadIdx.x; i < ng; i += B) {
        int cf = group_cfield[g0 + i];
        if (!WKE_GUARD(cf >= 0 && cf < K, kChkProductsSlot)) cf = 0;
        ctab[i] = cf * B;
    }
    cp_async_wait<0>();
    __syncthreads();
    const int ppg = PPGC > 0 ? PPGC : PPG;
    const int col = col0 + threadIdx.x;
    // this point's table offsets and signs: 3D V_1 at i3 (sign (-1)^{i2}) and
    // V_2 at i2 (sign (-1)^{i3}); 2D V_1 (sign (-1)^{col})
    int o1 = 0, o2 = 0;
    T s1, s2 = (T)0;
    if (d == 3) {
        const int i2 = col / N, i3 = col - i2 * N;
        o1 = i3;
        o2 = N + i2 - i2lo;
        s1 = (i2 & 1) ? (T)-1 : (T)1;
        s2 = (i3 & 1) ? (T)-1 : (T)1;
    } else {
        s1 = (col & 1) ? (T)-1 : (T)1;
    }
    const T sgn1 = (i1 & 1) ? (T)-1 : (T)1;
    cx<T> *fb = fbase + threadIdx.x;
    const cx<T> *tv = tabs;
    for (int u = 0; u < U; ++u, tv += TS) {
        const cx<T> Z = fb[(2 * u) * B];
        T a = (T)0, b = (T)0;
        if (NYQ) {
            const cx<T> v0 = fb[(2 * u + 1) * B], v1 = tv[o1];
            a = sgn1 * v0.x + s1 * v1.x;
            b = sgn1 * v0.y + s1 * v1.y;
            if (d == 3) {
                const cx<T> v2 = tv[o2];
                a += s2 * v2.x;
                b += s2 * v2.y;
            }
        }
        fb[(2 * u) * B] = mkc<T>(Z.x + b, a);
        if (2 * u + 1 < K) fb[(2 * u + 1) * B] = mkc<T>(Z.y - a, b);
    }
    const unsigned idx = p0 + threadIdx.x;
    const T F = f[idx];
    T sum = (T)0, comp = (T)0, sumi = (T)0, compi = (T)0;
    const ProdEntry<T> *pe = ptab;
    for (int g = 0; g < ng; ++g) {
        const cx<T> C = fb[ctab[g]];
        const T sr = C.x + F, si = C.y, cr = C.x * F, ci = C.y * F;
        T acc = (T)0, acci = (T)0;
#pragma unroll
        for (int p = 0; p < ppg; ++p, ++pe) {
            const ProdEntry<T> e = *pe;
            const cx<T> A = fb[e.ab & 0xffffu], Bf = fb[e.ab >> 16];
            const T pr = A.x * Bf.x - A.y * Bf.y, pim = A.x * Bf.y + A.y * Bf.x;   // A B
            const cx<T> Sab = cadd<T>(A, Bf);                                      // A + B
            const T ur = Sab.x, ui = Sab.y;
            acc += e.w * ((pr * sr - pim * si) - (cr * ur - ci * ui));
            if (IM) acci += e.w * ((pr * si + pim * sr) - (cr * ui + ci * ur));
        }
        T tsum = sum + acc;
        comp += fabs(sum) >= fabs(acc) ? (sum - tsum) + acc : (acc - tsum) + sum;
        sum = tsum;
        if (IM) {
            tsum = sumi + acci;
            compi += fabs(sumi) >= fabs(acci) ? (sumi - tsum) + acci : (acci - tsum) + sumi;
            sumi = tsum;
        }
    }
    Qacc[idx] += (double)sum + (double)comp;
    if (IM) Qim[idx] += (double)sumi + (double)compi;
}

// Fused axis-0 transform and product pass (3D, FP32, shared-field layout).
// Block: CB = LPW consecutive columns of one i2 row (LPW = lines per warp of
// the warp-line transform), all N points of each along axis 0, so N * CB
// points and as many threads.  Each warp takes whole units: its lanes hold
// the CB columns' lines (lane = column + CB * t), it forms the unit's axis-0
// input (the pass-1 output, or for separable plans E0a S_a + i E0b S_b from
// the pair planes), transforms it with the warp-local Stockham line
// (exchanges through the warp's own padded scratch, __syncwarp only), adds
// the Nyquist imaginary parts and writes the unit's two fields at its points
// into the block's field slots.  After one barrier every thread forms, at
// its point, the products of all groups of the chunk from the field slots,
// with the same algebra and summation order as k_products_staged.  The
// chunk's product table arrives as a kernel parameter.
// Add a point's chunk total (sum, comp: a compensated sum) to its
// accumulator; in the last chunk of an evaluation (Qout not null) write
// Q = scale * total instead (and Im Q when Qiout is not null) and clear the
// accumulators for the next evaluation, which is what the finalize kernel
// does for the other layouts.  FP64 plans keep one double per point.  FP32
// plans keep a float pair (hi, lo) in the same 8 bytes: hi takes the chunk
// totals by Neumaier's compensated addition and lo gathers the rounding
// errors and the chunks' compensations, so hi + lo carries about twice the
// FP32 significand over the chunks; no FP64 instruction is needed.
__device__ __forceinline__ float2 pair_add(float2 a, float s, float c) {
    const float t = a.x + s;
    const float e = fabsf(a.x) >= fabsf(s) ? (a.x - t) + s : (s - t) + a.x;
    return make_float2(t, a.y + (e + c));
}

template <typename T>
__device__ __forceinline__ void fused_epilogue(double *__restrict__ Qacc, double *__restrict__ Qim, size_t idx, T sum,
                                               T comp, T sumi, T compi, bool im, T *__restrict__ Qout,
                                               T *__restrict__ Qiout, double scale) {
    if constexpr (sizeof(T) == 4) {
        float2 *A = reinterpret_cast<float2 *>(Qacc), *Ai = reinterpret_cast<float2 *>(Qim);
        const float2 a = pair_add(A[idx], sum, comp);
        if (Qout) {
            Qout[idx] = (float)scale * (a.x + a.y);      // scale is a power of two
            A[idx] = make_float2(0.f, 0.f);
        } else {
            A[idx] = a;
        }
        if (im) {
            const float2 ai = pair_add(Ai[idx], sumi, compi);
            if (Qout) {
                if (Qiout) Qiout[idx] = (float)scale * (ai.x + ai.y);
                Ai[idx] = make_float2(0.f, 0.f);
            } else {
                Ai[idx] = ai;
            }
        }
    } else {
        const double add = (double)sum + (double)comp, add_im = (double)sumi + (double)compi;
        if (Qout) {
            Qout[idx] = (T)(scale * (Qacc[idx] + add));
            Qacc[idx] = 0.0;
            if (im) {
                if (Qiout) Qiout[idx] = (T)(scale * (Qim[idx] + add_im));
                Qim[idx] = 0.0;
            }
        } else {
            Qacc[idx] += add;
            if (im) Qim[idx] += add_im;
        }
    }
}

template <typename T> struct FusedTab {
    static constexpr int kMaxProducts = 256, kMaxGroups = 64;
    unsigned char pa[kMaxProducts], pb[kMaxProducts];   // chunk-local field ids
    unsigned char cf[kMaxGroups];                       // C field of each group
    T w[kMaxProducts];
};

template <typename T, int N, bool SEP, bool IM, bool NYQ, int PPGC>
__global__ void __launch_bounds__(N * LineCfg<T, N>::LPW)
k_fused_3d(const cx<T> *__restrict__ src, const cx<T> *__restrict__ phase, const int *__restrict__ field_pair,
           const cx<T> *__restrict__ Vtab, const T *__restrict__ f, double *__restrict__ Qacc,
           double *__restrict__ Qim, const cx<T> *__restrict__ tw_g, int sf0, int K, int ng, int PPG,
           const __grid_constant__ FusedTab<T> tab, T *__restrict__ Qout, T *__restrict__ Qiout, double scale) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    constexpr int CB = LPW, PTS = N * CB, WARPS = PTS / 32;
    constexpr int P = N * N;
    constexpr size_t ND = (size_t)N * P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *fld = tw + N;                                   // field k at point pt: fld[k * PTS + pt]
    cx<T> *scr = fld + (size_t)K * PTS;                    // WARPS * LPW lines of LinePad<N>::PITCH
    const cx<T> twv = twiddle_fetch<T, N>(tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int col0 = blockIdx.x * CB;
    const int i2 = col0 / N, i3 = col0 - i2 * N + c;      // this lane's column (transform phase)
    const int col = col0 + c;
    const int U = (K + 1) / 2;
    twiddle_store<T, N>(tw, twv, tw_g);
    cx<T> *wscr = scr + (size_t)(warp * LPW + c) * LinePad<N>::PITCH;
    const T sgn1 = (t & 1) ? (T)-1 : (T)1;               // (-1)^{i1}: TPL is even
    const T s2 = (i2 & 1) ? (T)-1 : (T)1, s3 = (i3 & 1) ? (T)-1 : (T)1;
    for (int u = warp; u < U; u += WARPS) {
        const int fa = sf0 + 2 * u;
        const bool pair = 2 * u + 1 < K;
        cx<T> v[E];
        if (SEP) {
            const int fb = pair ? fa + 1 : fa;
            // the FP32 N = 64 planes are column-blocked (k_sep_planes64)
            const int scol = (N == 64 && sizeof(T) == 4) ? sep_col64(col) : col;
            const cx<T> *sa = src + (size_t)field_pair[fa] * ND + scol, *sb = src + (size_t)field_pair[fb] * ND + scol;
            const cx<T> *ea = phase + (size_t)fa * 3 * N, *eb = phase + (size_t)fb * 3 * N;
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sep_input<T>(sa, sb, ea, eb, t + e * TPL, P, pair);
        } else {
            const cx<T> *hu = src + (size_t)u * ND + col;
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = hu[(size_t)(t + e * TPL) * P];
        }
        // Nyquist imaginary parts (a of the real-slot field, b of the other)
        cx<T> nq[E];
        if (NYQ) {
            const cx<T> *Vu = Vtab + (size_t)u * 3 * P;
            const cx<T> v0 = Vu[col];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i1 = t + e * TPL;
                const cx<T> v1 = Vu[P + i1 * N + i3], v2 = Vu[2 * P + i1 * N + i2];
                nq[e] = mkc<T>(sgn1 * v0.x + s2 * v1.x + s3 * v2.x, sgn1 * v0.y + s2 * v1.y + s3 * v2.y);
            }
        }
        line_fft<T, N, E, +1>(v, t, wscr, tw);
        cx<T> *fa_s = fld + (size_t)(2 * u) * PTS + c;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pt = (t + e * TPL) * CB;
            const T a = NYQ ? nq[e].x : (T)0, b = NYQ ? nq[e].y : (T)0;
            fa_s[pt] = mkc<T>(v[e].x + b, a);
            if (pair) fa_s[PTS + pt] = mkc<T>(v[e].y - a, b);
        }
    }
    __syncthreads();
    // products at this thread's point
    const int pt = threadIdx.x;
    const int i1 = pt / CB, zc = pt - i1 * CB;
    const size_t idx = (size_t)i1 * P + col0 + zc;
    const cx<T> *fb = fld + pt;
    const T F = f[idx];
    const int ppg = PPGC > 0 ? PPGC : PPG;
    T sum = (T)0, comp = (T)0, sumi = (T)0, compi = (T)0;
    int k = 0;
    for (int g = 0; g < ng; ++g) {
        const cx<T> C = fb[(int)tab.cf[g] * PTS];
        const T sr = C.x + F, si = C.y, cr = C.x * F, ci = C.y * F;
        T acc = (T)0, acci = (T)0;
#pragma unroll
        for (int p = 0; p < ppg; ++p, ++k) {
            const cx<T> A = fb[(int)tab.pa[k] * PTS], Bf = fb[(int)tab.pb[k] * PTS];
            const T w = tab.w[k];
            const T pr = A.x * Bf.x - A.y * Bf.y, pim = A.x * Bf.y + A.y * Bf.x;   // A B
            const cx<T> Sab = cadd<T>(A, Bf);                                      // A + B
            const T ur = Sab.x, ui = Sab.y;
            acc += w * ((pr * sr - pim * si) - (cr * ur - ci * ui));
            if (IM) acci += w * ((pr * si + pim * sr) - (cr * ui + ci * ur));
        }
        T tsum = sum + acc;
        comp += fabs(sum) >= fabs(acc) ? (sum - tsum) + acc : (acc - tsum) + sum;
        sum = tsum;
        if (IM) {
            tsum = sumi + acci;
            compi += fabs(sumi) >= fabs(acci) ? (sumi - tsum) + acci : (acci - tsum) + sumi;
            sumi = tsum;
        }
    }
    fused_epilogue<T>(Qacc, Qim, idx, sum, comp, sumi, compi, IM, Qout, Qiout, scale);
}

// Fused axis-0 transform and product pass for N = 64 in FP32.  A block holds
// 4 consecutive columns of one i2 row (256 points, 256 threads) and one slot
// of 256 points per unit, its two fields interleaved (16 bytes per point).
// It first copies with cp.async its columns of the chunk's pair planes
// (separable plans) or of the pass-1 units into shared memory, then each
// warp transforms whole units: the axis-0 input from the staged columns
// (and, separable, the fields' axis-0 phases), the line transform with the
// exchange of line64_swz in the first half of the unit's slot, and the
// unpacking of both fields into the slot (one 16-byte store per point) with
// the Nyquist imaginary parts, whose table entries the warp loads from L2
// before the transform.
// After one barrier every thread forms the products at its point with the
// algebra and summation order of k_fused_3d.  The chunk's product schedule
// arrives as a kernel parameter with shared-memory byte offsets, so that
// with the group count a template constant (NGC > 0) every offset and weight
// is an immediate operand.  When the products of every group share one
// weight (EQW; the equal-weight rules of Sec. 3.3), a group's sum is formed as
//   w Re[s P - cf U],  P = sum_p A_p B_p,  U = sum_p (A_p + B_p),
// the same sum as the per-product form with the weight and the factors s
// and cf taken out of the product loop.
constexpr int kF64Pts = 256;

struct Fused64Tab {
    static constexpr int kMaxProducts = 256, kMaxGroups = 64, kMaxUnits = 128;
    unsigned oa[kMaxProducts], ob[kMaxProducts];   // byte offsets of each product's fields from the
                                                   // point's unit entry: (l / 2) 256 * 16 + (l % 2) 8
    unsigned oc[kMaxGroups];                       // byte offset of each group's C field
    float w[kMaxProducts];
    unsigned char pla[kMaxUnits], plb[kMaxUnits];  // separable plans: pair plane of each unit's fields
};

// P += A B, U += A + B (complex).
__device__ __forceinline__ void pu_acc(float2 &P, float2 &U, float2 A, float2 B) {
    P.x = fmaf(A.x, B.x, P.x);
    P.x = fmaf(-A.y, B.y, P.x);
    P.y = fmaf(A.x, B.y, P.y);
    P.y = fmaf(A.y, B.x, P.y);
    U = cadd<float>(U, cadd<float>(A, B));
}

// CUBE: the cube rule's schedule (3 products per group, 8 groups, one weight
// per group) on a chunk whose 26 fields the plan ordered as the edge fields
// (field 2 i + s: axis i, s = 1 negative), the face fields (6 + 4 i + q: the
// face with component i zero, q's bit 0 the lower other axis negative, bit 1
// the higher one) and the C fields (18 + v: the group of vertex v, bit a:
// v_a < 0); tab.w[v] is the weight of the group of vertex v.
template <bool SEP, bool IM, bool NYQ, int PPGC, int NGC, bool EQW, bool CUBE>
__global__ void __launch_bounds__(256, 3)
k_fused64(const float2 *__restrict__ src, const float4 *__restrict__ ue0, const float2 *__restrict__ Vtab,
          const float *__restrict__ f, double *__restrict__ Qacc, double *__restrict__ Qim,
          const float2 *__restrict__ tw_g, int K, int ng, int PPG, int nplanes, int ubase,
          const __grid_constant__ Fused64Tab tab, float *__restrict__ Qout, float *__restrict__ Qiout,
          double scale) {
    constexpr int N = 64, CB = 4, PTS = kF64Pts, P = N * N;
    constexpr size_t ND = (size_t)N * P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int U = (K + 1) / 2;
    // unit u's two fields interleaved: field 2u + h of point pt at float2
    // index (u PTS + pt) 2 + h, so that one 16-byte access covers both
    float2 *fld = reinterpret_cast<float2 *>(smem_raw);             // U unit slots of PTS points
    float2 *pst = fld + (size_t)2 * U * PTS;                          // staged planes: [plane][j1][c]
    float2 *tws = pst + (size_t)nplanes * PTS;                        // twiddles exp(2 pi i k / 64)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = lane & 3, t = lane >> 2;
    const int col0 = blockIdx.x * CB;
    const int i2 = col0 >> 6, i30 = col0 & 63;
    // ---- stage the planes: 128 pieces of 16 bytes per plane, two planes per pass
    {
        const int j1 = (tid >> 1) & 63, h = tid & 1;
        // separable plans: column-blocked pair planes (sep_col64); pass-1 units: row-major
        const float2 *sp = src + (size_t)j1 * P + (SEP ? sep_col64(col0) : col0) + 2 * h;
        float2 *dp = pst + j1 * CB + 2 * h;
        for (int pl = tid >> 7; pl < nplanes; pl += 2) cp_async16(dp + (size_t)pl * PTS, sp + (size_t)pl * ND);
    }
    cp_async_commit();
    if (tid < N) tws[tid] = tw_g[tid];
    const float sgn1 = (t & 1) ? -1.0f : 1.0f;                         // (-1)^{i1}
    const float s2 = (i2 & 1) ? -1.0f : 1.0f, s3 = ((i30 + c) & 1) ? -1.0f : 1.0f;
    cp_async_wait<0>();
    __syncthreads();
    for (int u = warp; u < U; u += 8) {
        const bool pair = 2 * u + 1 < K;
        // this thread's Nyquist-table entries of unit u (from L2, in flight
        // during the transform)
        float2 vr[17];
        if (NYQ) {
            const float2 *Vu = Vtab + (size_t)u * 3 * P;
            vr[16] = Vu[col0 + c];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                vr[e] = Vu[P + (t + 8 * e) * N + i30 + c];
                vr[8 + e] = Vu[2 * P + (t + 8 * e) * N + i2];
            }
        }
        float2 v[8];
        if (SEP && !WKE_GUARD(tab.pla[u] < nplanes && tab.plb[u] < nplanes, kChkFusedPlane)) continue;
        if (!SEP && !WKE_GUARD(u < nplanes, kChkFusedPlane)) continue;
        if (SEP) {
            const float2 *sa = pst + (size_t)tab.pla[u] * PTS + c, *sb = pst + (size_t)tab.plb[u] * PTS + c;
            const float4 *e0 = ue0 + (size_t)(ubase + u) * N;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j1 = t + 8 * e;
                const float4 ph = e0[j1];
                const float2 A = cmul<float>(sa[j1 * CB], make_float2(ph.x, ph.y));
                const float2 B = cmul<float>(sb[j1 * CB], make_float2(ph.z, ph.w));
                v[e] = make_float2(A.x - B.y, A.y + B.x);
            }
        } else {
            const float2 *hu = pst + (size_t)u * PTS + c;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = hu[(t + 8 * e) * CB];
        }
        float2 *slot = fld + (size_t)(2 * u) * PTS;
        line64_swz(v, c, t, slot, tws);
        const float2 v0 = NYQ ? vr[16] : make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int pt = (t + 8 * e) * CB + c;
            float a = 0.f, b = 0.f;
            if (NYQ) {
                a = sgn1 * v0.x + s2 * vr[e].x + s3 * vr[8 + e].x;
                b = sgn1 * v0.y + s2 * vr[e].y + s3 * vr[8 + e].y;
            }
            if (pair)
                *reinterpret_cast<float4 *>(slot + 2 * pt) = make_float4(v[e].x + b, a, v[e].y - a, b);
            else
                slot[2 * pt] = make_float2(v[e].x + b, a);
        }
    }
    __syncthreads();
    // ---- products at this thread's point
    const int pt = tid;
    const size_t idx = (size_t)(pt >> 2) * P + col0 + (pt & 3);
    const unsigned char *fb = reinterpret_cast<const unsigned char *>(fld + 2 * pt);
    // checked builds: a schedule offset outside the U unit slots reads slot 0
    const unsigned olim = (unsigned)U * PTS * sizeof(float4);
    auto off = [&](unsigned o) -> unsigned { return WKE_GUARD(o < olim, kChkFusedSchedule) ? o : 0u; };
    const float F = f[idx];
    const int ppg = PPGC > 0 ? PPGC : PPG;
    const int ngr = NGC > 0 ? NGC : ng;
    float sum = 0.f, comp = 0.f, sumi = 0.f, compi = 0.f;
    if constexpr (CUBE) {
        // axis by axis: the two edge fields of axis i meet its four face
        // fields, each pair a product of the vertex they agree with, so that
        // every field is read once per point; P = sum A B and U = sum (A + B)
        // per group in registers.  The plan orders the chunk's fields so that
        // unit i holds the edges of axis i (+, -), units 3 + 2i and 4 + 2i its
        // faces (q = 0, 1 and 2, 3) and units 9 + v/2 the C fields of the
        // vertices, so each load takes the two fields of one unit.
        constexpr unsigned kUnit = PTS * sizeof(float4);
        const bool ok = WKE_GUARD(K == 26, kChkFusedSchedule);
        auto unit2 = [&](int u) -> float4 {
            return ok ? *reinterpret_cast<const float4 *>(fb + u * kUnit) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        // (axis 0 sets every vertex's P and U, axes 1 and 2 add to them)
        float2 Pq[8], Uq[8];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = i == 0 ? 1 : 0, k = i == 2 ? 1 : 2;
            const float4 E2 = unit2(i);
            const float2 Ep = make_float2(E2.x, E2.y), Em = make_float2(E2.z, E2.w);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 F2 = unit2(3 + 2 * i + h);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = 2 * h + r;
                    const float2 Fc = r ? make_float2(F2.z, F2.w) : make_float2(F2.x, F2.y);
                    const int vp = ((q & 1) << j) | ((q >> 1) << k), vm = vp | (1 << i);
                    if (i == 0) {
                        Pq[vp] = cmul<float>(Ep, Fc);
                        Uq[vp] = cadd<float>(Ep, Fc);
                        Pq[vm] = cmul<float>(Em, Fc);
                        Uq[vm] = cadd<float>(Em, Fc);
                    } else {
                        pu_acc(Pq[vp], Uq[vp], Ep, Fc);
                        pu_acc(Pq[vm], Uq[vm], Em, Fc);
                    }
                }
            }
        }
        // the groups of vertices 2n and 2n + 1 (one C-field unit) are added
        // plainly and their sum enters the compensated running sum
        float pr = 0.f, pri = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const float4 C2 = unit2(9 + v / 2);
            const float2 C = (v & 1) ? make_float2(C2.z, C2.w) : make_float2(C2.x, C2.y);
            const float sr = C.x + F, si = C.y, cr = C.x * F, ci = C.y * F;
            const float w = tab.w[v];
            const float acc = w * ((sr * Pq[v].x - si * Pq[v].y) - (cr * Uq[v].x - ci * Uq[v].y));
            const float acci = IM ? w * ((sr * Pq[v].y + si * Pq[v].x) - (cr * Uq[v].y + ci * Uq[v].x)) : 0.f;
            if ((v & 1) == 0) {
                pr = acc;
                pri = acci;
                continue;
            }
            const float a = pr + acc;
            float tsum = sum + a;
            comp += fabsf(sum) >= fabsf(a) ? (sum - tsum) + a : (a - tsum) + sum;
            sum = tsum;
            if (IM) {
                const float ai = pri + acci;
                tsum = sumi + ai;
                compi += fabsf(sumi) >= fabsf(ai) ? (sumi - tsum) + ai : (ai - tsum) + sumi;
                sumi = tsum;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < (CUBE ? 0 : ngr); ++g) {
        const float2 C = *reinterpret_cast<const float2 *>(fb + off(tab.oc[g]));
        const float sr = C.x + F, si = C.y, cr = C.x * F, ci = C.y * F;
        float acc = 0.f, acci = 0.f;
        if (EQW) {
            // P = sum A B, U = sum (A + B); the group's weight once
            float2 Pq = make_float2(0.f, 0.f), Uq = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < ppg; ++p) {
                const int k = g * ppg + p;
                const float2 A = *reinterpret_cast<const float2 *>(fb + off(tab.oa[k]));
                const float2 Bf = *reinterpret_cast<const float2 *>(fb + off(tab.ob[k]));
                Pq.x = fmaf(A.x, Bf.x, Pq.x);
                Pq.x = fmaf(-A.y, Bf.y, Pq.x);
                Pq.y = fmaf(A.x, Bf.y, Pq.y);
                Pq.y = fmaf(A.y, Bf.x, Pq.y);
                Uq = cadd<float>(Uq, cadd<float>(A, Bf));
            }
            const float w = tab.w[g * ppg];
            acc = w * ((sr * Pq.x - si * Pq.y) - (cr * Uq.x - ci * Uq.y));
            if (IM) acci = w * ((sr * Pq.y + si * Pq.x) - (cr * Uq.y + ci * Uq.x));
        } else {
#pragma unroll
            for (int p = 0; p < ppg; ++p) {
                const int k = g * ppg + p;
                const float2 A = *reinterpret_cast<const float2 *>(fb + off(tab.oa[k]));
                const float2 Bf = *reinterpret_cast<const float2 *>(fb + off(tab.ob[k]));
                const float w = tab.w[k];
                const float pr = A.x * Bf.x - A.y * Bf.y, pim = A.x * Bf.y + A.y * Bf.x;   // A B
                const float2 Sab = cadd<float>(A, Bf);                                   // A + B
                acc += w * ((pr * sr - pim * si) - (cr * Sab.x - ci * Sab.y));
                if (IM) acci += w * ((pr * si + pim * sr) - (cr * Sab.y + ci * Sab.x));
            }
        }
        float tsum = sum + acc;
        comp += fabsf(sum) >= fabsf(acc) ? (sum - tsum) + acc : (acc - tsum) + sum;
        sum = tsum;
        if (IM) {
            tsum = sumi + acci;
            compi += fabsf(sumi) >= fabsf(acci) ? (sumi - tsum) + acci : (acci - tsum) + sumi;
            sumi = tsum;
        }
    }
    fused_epilogue<float>(Qacc, Qim, idx, sum, comp, sumi, compi, IM, Qout, Qiout, scale);
}

// ------------------------------------------------------------------ finalize
// Q = scale * sum_g Qacc[g] in group order; the accumulators are cleared.
template <typename T>
__global__ void k_finalize(double *__restrict__ Qacc, double *__restrict__ Qim, int G, size_t ND, double scale,
                           T *__restrict__ Q, T *__restrict__ Qi) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) {
            s += Qacc[g * ND + i];
            Qacc[g * ND + i] = 0.0;
        }
        Q[i] = (T)(scale * s);
        if (Qim) {
            double si = 0.0;
            for (int g = 0; g < G; ++g) {
                si += Qim[g * ND + i];
                Qim[g * ND + i] = 0.0;
            }
            if (Qi) Qi[i] = (T)(scale * si);
        }
    }
}

// Finalize of the FP32 fused layouts' (hi, lo) accumulator pairs (one
// accumulator): Q = scale * (hi + lo) into a double grid; the pairs are
// cleared.
template <typename TQ>
__global__ void k_finalize_pair(double *__restrict__ Qacc, size_t ND, double scale, TQ *__restrict__ Q) {
    float2 *A = reinterpret_cast<float2 *>(Qacc);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = A[i];
        Q[i] = (TQ)(scale * ((double)a.x + (double)a.y));
        A[i] = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------ de-aliasing (2N grid)
// Coefficients of f on the 2N grid: mode j of [-Nin/2, Nin/2-1]^d keeps its
// value, the other modes of [-N/2, N/2-1]^d (N = 2 Nin) are zero.  Both
// arrays in DFT order.
template <typename T>
__global__ void k_pad_spectrum(const cx<T> *__restrict__ gin, cx<T> *__restrict__ g, int d, int Nin, int N,
                               size_t ND) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x) {
        size_t rest = i, src = 0, stride = 1;
        bool inside = true;
        for (int a = d - 1; a >= 0; --a) {
            const int pos = (int)(rest % N);
            rest /= N;
            const int j = pos < N / 2 ? pos : pos - N;       // signed mode on the 2N grid
            if (j < -Nin / 2 || j >= Nin / 2) inside = false;
            src += (size_t)(j < 0 ? j + Nin : j) * stride;  // its position on the Nin grid
            stride *= Nin;
        }
        g[i] = inside ? gin[src] : mkc<T>((T)0, (T)0);
    }
}

// One axis of a separable linear map in double: out[a][i][b] =
// sum_{i'} K[i][i'] in[a][i'][b] for a < A, i < n_out, b < B.  Inputs are
// real (float or double) or complex (double2); outputs complex (double2) or
// real parts in `out` and imaginary parts in `out_im` (if not null).
__device__ __forceinline__ double2 as_cx(float v) { return make_double2((double)v, 0.0); }
__device__ __forceinline__ double2 as_cx(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double2 as_cx(double2 v) { return v; }
__device__ __forceinline__ void put_cx(double2 *out, double2 *, size_t i, double2 v) { out[i] = v; }
template <typename T> __device__ __forceinline__ void put_cx(T *out, T *out_im, size_t i, double2 v) {
    out[i] = (T)v.x;
    if (out_im) out_im[i] = (T)v.y;
}

template <typename TIn, typename TOut>
__global__ void k_axis_map(const TIn *__restrict__ in, TOut *__restrict__ out, TOut *__restrict__ out_im,
                           const double2 *__restrict__ K, int n_out, int n_in, size_t A, size_t B) {
    const size_t total = A * (size_t)n_out * B;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t b = idx % B, r = idx / B;
        const int i = (int)(r % n_out);
        const size_t a = r / n_out;
        const double2 *Kr = K + (size_t)i * n_in;
        const TIn *src = in + a * n_in * B + b;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < n_in; ++k) {
            const double2 x = as_cx(src[(size_t)k * B]);
            const double2 w = Kr[k];
            re += w.x * x.x - w.y * x.y;
            im += w.x * x.y + w.y * x.x;
        }
        put_cx(out, out_im, idx, make_double2(re, im));
    }
}

// ------------------------------------------------------------------ moments
// Per-block partial sums of h^d [g, k g, |k|^2 g] in double; a second
// single-block kernel adds the partials in block order (deterministic).
constexpr int kMomentBlocks = 256;
constexpr int kMomentThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kMomentThreads)
k_moments(const T *__restrict__ g, int d, int N, double L, double *__restrict__ partials) {
    const size_t ND = d == 2 ? (size_t)N * N : (size_t)N * N * N;
    const double h = 2.0 * L / N;
    double acc[5] = {0, 0, 0, 0, 0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)g[i];
        size_t rest = i;
        double k2 = 0.0;
        double kk[3] = {0, 0, 0};
        for (int a = d - 1; a >= 0; --a) {
            const double ka = -L + (double)(rest % N) * h;
            rest /= N;
            kk[a] = ka;
            k2 += ka * ka;
        }
        acc[0] += v;
        for (int a = 0; a < d; ++a) acc[1 + a] += kk[a] * v;
        acc[d + 1] += k2 * v;
    }
    __shared__ double red[5][kMomentThreads];
    for (int k = 0; k < d + 2; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kMomentThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < d + 2; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < d + 2; ++k) partials[blockIdx.x * (d + 2) + k] = red[k][0];
}

static __global__ void k_moments_reduce(const double *__restrict__ partials, int nblocks, int K, double hd,
                                 double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k < K) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * K + k];
        out[k] = hd * s;
    }
}

// ------------------------------------------------------------------ Runge-Kutta
// kacc (+)= b_s k; ystage = f + c_next dt k (skipped when c_next_dt is 0 and
// ystage is null).
template <typename T>
__global__ void k_rk_stage(const T *__restrict__ f, const T *__restrict__ k, double *__restrict__ kacc,
                           T *__restrict__ ystage, double b_s, double c_next_dt, int first, size_t ND) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x) {
        const double kv = (double)k[i];
        kacc[i] = first ? b_s * kv : kacc[i] + b_s * kv;
        if (ystage) ystage[i] = (T)((double)f[i] + c_next_dt * kv);
    }
}

template <typename T>
__global__ void k_rk_final(T *__restrict__ f, const double *__restrict__ kacc, double dt, size_t ND) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ND; i += (size_t)gridDim.x * blockDim.x)
        f[i] = (T)((double)f[i] + dt * kacc[i]);
}

}  // namespace wke
