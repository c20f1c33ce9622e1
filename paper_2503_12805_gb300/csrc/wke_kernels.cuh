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

template <typename T, int N>
__device__ __forceinline__ void load_twiddles(cx<T> *tw, const cx<T> *tw_g) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();
}

// ------------------------------------------------------------------ forward
// 3D: forward transform over axes (1, 2) of every plane i1 of the real input,
// in double.  One block per plane: row lines along axis 2, then column lines
// along axis 1 with consecutive columns per warp (coalesced stores).
template <typename TIn, int N>
__global__ void __launch_bounds__(N * LineCfg<double, N>::TPL)
k_fwd_planes_3d(const TIn *__restrict__ f, double2 *__restrict__ tmp, const double2 *__restrict__ tw_g) {
    typedef LineCfg<double, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, WP = Work<N>::PITCH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tw = reinterpret_cast<double2 *>(smem_raw);
    double2 *work = tw + N;
    double2 *scratch = work + N * WP;
    load_twiddles<double, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int row = warp * LPW + c;
    const int z = threadIdx.x % N, ty = threadIdx.x / N;
    double2 *rscr = scratch + (size_t)row * LinePad<N>::PITCH;
    const int i1 = blockIdx.x;
    const TIn *src = f + ((size_t)i1 * N + row) * N;
    double2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = make_double2((double)src[t + e * TPL], 0.0);
    line_fft<double, N, E, -1>(v, t, rscr, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) work[row * WP + t + e * TPL] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = work[(ty + e * TPL) * WP + z];
    col_fft<double, N, E, -1>(v, ty, scratch, z, N, tw);
    double2 *out = tmp + (size_t)i1 * N * N;
#pragma unroll
    for (int e = 0; e < E; ++e) out[(ty + e * TPL) * N + z] = v[e];
}

// 2D: forward transform of every row, in double.
template <typename TIn, int N>
__global__ void k_fwd_rows_2d(const TIn *__restrict__ f, double2 *__restrict__ tmp, const double2 *__restrict__ tw_g) {
    typedef LineCfg<double, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tw = reinterpret_cast<double2 *>(smem_raw);
    double2 *scratch = tw + N;
    load_twiddles<double, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    const int i1 = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    double2 *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    double2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = make_double2((double)f[(size_t)i1 * N + t + e * TPL], 0.0);
    line_fft<double, N, E, -1>(v, t, scr, tw);
#pragma unroll
    for (int e = 0; e < E; ++e) tmp[(size_t)i1 * N + t + e * TPL] = v[e];
}

// Both d: forward transform along axis 0 of every column; writes
// ghat = DFT / N^d in T, optionally zeroing modes with a component -N/2.
template <typename TOut, int N>
__global__ void k_fwd_cols(const double2 *__restrict__ tmp, cx<TOut> *__restrict__ ghat,
                           const double2 *__restrict__ tw_g, int P, int d, double inv_nd, int nyq_zero) {
    typedef LineCfg<double, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tw = reinterpret_cast<double2 *>(smem_raw);
    double2 *scratch = tw + N;
    load_twiddles<double, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int wl = warp * LPW + c;
    const int col = blockIdx.x * (blockDim.x / 32) * LPW + wl;
    double2 *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    double2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = tmp[(size_t)(t + e * TPL) * P + col];
    line_fft<double, N, E, -1>(v, t, scr, tw);
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
        double2 x = v[e];
        if (nyq_zero && (col_nyq || j1 == N / 2)) x = make_double2(0.0, 0.0);
        ghat[(size_t)j1 * P + col] = mkc<TOut>((TOut)(x.x * inv_nd), (TOut)(x.y * inv_nd));
    }
}

// ------------------------------------------------------------------ pass 1
// 3D: block (j1, field block).  For each field of the block: row lines take
// the phase-weighted spectrum of plane j1 and transform along axis 2 (one
// warp per LPW rows); the rows go through shared memory; then every column
// z is transformed along axis 1 by N/8 threads spread over the block, with
// 32 consecutive columns per warp, so the stores to H[field][j1][y][z] are
// whole 256-byte rows.
template <typename T, int N>
__global__ void __launch_bounds__(N * LineCfg<T, N>::TPL)
k_pass1_3d(const cx<T> *__restrict__ ghat, const cx<T> *__restrict__ phase, cx<T> *__restrict__ H,
           const cx<T> *__restrict__ tw_g, int field0, int nfields, int fields_per_block) {
    typedef LineCfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL, LPW = Cfg::LPW, WP = Work<N>::PITCH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *work = tw + N;
    cx<T> *scratch = work + N * WP;           // row scratch, then column scratch
    load_twiddles<T, N>(tw, tw_g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % LPW, t = lane / LPW;
    const int row = warp * LPW + c;           // axis-1 index j2 of this row line
    const int z = threadIdx.x % N, ty = threadIdx.x / N;   // column lines
    cx<T> *rscr = scratch + (size_t)row * LinePad<N>::PITCH;
    const int j1 = blockIdx.x;
    const int fbeg = blockIdx.y * fields_per_block;
    const int fend = min(nfields, fbeg + fields_per_block);
    const size_t NN = (size_t)N * N;
    const cx<T> *grow = ghat + ((size_t)j1 * N + row) * N;
    cx<T> g[E];
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = grow[t + e * TPL];
    for (int fl = fbeg; fl < fend; ++fl) {
        const cx<T> *ph = phase + (size_t)(field0 + fl) * 3 * N;
        const cx<T> p01 = cmul<T>(ph[j1], ph[N + row]);
        cx<T> v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmul<T>(cmul<T>(g[e], ph[2 * N + t + e * TPL]), p01);
        line_fft<T, N, E, +1>(v, t, rscr, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) work[row * WP + t + e * TPL] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = work[(ty + e * TPL) * WP + z];
        col_fft<T, N, E, +1>(v, ty, scratch, z, N, tw);
        cx<T> *out = H + ((size_t)fl * N + j1) * NN;
#pragma unroll
        for (int e = 0; e < E; ++e) out[(ty + e * TPL) * N + z] = v[e];
        __syncthreads();
    }
}

// 2D: block (row block, field).  Row j1 of the phase-weighted spectrum,
// inverse transform along axis 1 -> H[field][j1][y].
template <typename T, int N>
__global__ void k_pass1_2d(const cx<T> *__restrict__ ghat, const cx<T> *__restrict__ phase, cx<T> *__restrict__ H,
                           const cx<T> *__restrict__ tw_g, int field0) {
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
    const int fl = blockIdx.y;
    cx<T> *scr = scratch + (size_t)wl * LinePad<N>::PITCH;
    const cx<T> *ph = phase + (size_t)(field0 + fl) * 2 * N;
    const cx<T> p0 = ph[j1];
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; ++e)
        v[e] = cmul<T>(cmul<T>(ghat[(size_t)j1 * N + t + e * TPL], ph[N + t + e * TPL]), p0);
    line_fft<T, N, E, +1>(v, t, scr, tw);
    cx<T> *out = H + ((size_t)fl * N + j1) * N;
#pragma unroll
    for (int e = 0; e < E; ++e) out[t + e * TPL] = v[e];
}

// ------------------------------------------------------------------ pass 2
// Block (column tile, group of the chunk).  A tile is CB consecutive columns
// of the trailing axes; each column's N points along axis 0 are held by
// TPL = N/E threads spread over the block (thread ty holds points
// ty + e TPL), so every warp reads and writes 32 consecutive columns of one
// row.  The block transforms C once and keeps s = C + F and cf = C F; for
// every product of the group it transforms A, forms X = A s - cf and adds
// the term -cf A, then transforms B and adds B X, since
// A B (C + F) - C F (A + B) = B (A s - cf) - cf A.  Only one transformed
// field is live at a time.  The group's sum goes to that group's double
// accumulator.
template <typename T, int N> struct Pass2Cfg {
    static constexpr int E = N <= 64 ? 4 : 8;           // points per thread
    static constexpr int TPL = N / E;                    // threads per column
    static constexpr int THREADS = 256;
    static constexpr int CB = THREADS / TPL;             // columns per block (at most)
    static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? (E == 4 ? 3 : 2) : (E == 4 ? 2 : 1);
};

template <typename T, int N, bool IM>
__global__ void __launch_bounds__(Pass2Cfg<T, N>::THREADS, Pass2Cfg<T, N>::MIN_BLOCKS)
k_pass2(const cx<T> *__restrict__ H, const T *__restrict__ f, double *__restrict__ Qacc, double *__restrict__ Qim,
        const int *__restrict__ prod_local, const double *__restrict__ prod_W, const cx<T> *__restrict__ tw_g, int P,
        int CB, int FPG, int PPG, int g0) {
    typedef Pass2Cfg<T, N> Cfg;
    constexpr int E = Cfg::E, TPL = Cfg::TPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *tw = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *scratch = tw + N;                  // LinePad<N>::LEN rows x CB columns
    load_twiddles<T, N>(tw, tw_g);
    const int z = threadIdx.x % CB, t = threadIdx.x / CB;
    const int col = blockIdx.x * CB + z;
    const int gl = blockIdx.y;
    const size_t ND = (size_t)N * P;
    const cx<T> *Hg = H + (size_t)gl * FPG * ND;

    cx<T> v[E], s[E], cf[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = Hg[(size_t)(t + e * TPL) * P + col];
    col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
    T ar[E], ai[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const T F = f[(size_t)(t + e * TPL) * P + col];
        s[e] = mkc<T>(v[e].x + F, v[e].y);
        cf[e] = mkc<T>(v[e].x * F, v[e].y * F);
        ar[e] = (T)0;
        ai[e] = (T)0;
    }
    const double *Wg = prod_W + (size_t)(g0 + gl) * PPG;
    for (int p = 0; p < PPG; ++p) {
        const cx<T> *HA = Hg + (size_t)prod_local[2 * p] * ND;
        const cx<T> *HB = Hg + (size_t)prod_local[2 * p + 1] * ND;
        const T W = (T)Wg[p];
        cx<T> X[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = HA[(size_t)(t + e * TPL) * P + col];
        col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            X[e] = csub<T>(cmul<T>(v[e], s[e]), cf[e]);
            const cx<T> q = cmul<T>(cf[e], v[e]);            // added with a minus sign
            ar[e] -= W * q.x;
            if (IM) ai[e] -= W * q.y;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = HB[(size_t)(t + e * TPL) * P + col];
        col_fft<T, N, E, +1>(v, t, scratch, z, CB, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            ar[e] += W * (v[e].x * X[e].x - v[e].y * X[e].y);
            if (IM) ai[e] += W * (v[e].x * X[e].y + v[e].y * X[e].x);
        }
    }
    double *Qg = Qacc + (size_t)gl * ND;
#pragma unroll
    for (int e = 0; e < E; ++e) Qg[(size_t)(t + e * TPL) * P + col] += (double)ar[e];
    if (IM) {
        double *Qig = Qim + (size_t)gl * ND;
#pragma unroll
        for (int e = 0; e < E; ++e) Qig[(size_t)(t + e * TPL) * P + col] += (double)ai[e];
    }
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
