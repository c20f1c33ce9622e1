// Launch wrappers for one real type T; included by the per-precision
// translation units, which instantiate them explicitly.
#pragma once

#include <algorithm>

#include "wke_kernels.cuh"

namespace wke {

template <typename K> static int set_smem(K kernel, size_t bytes) {
    if (int rc = check_bind()) return rc;   // checked builds: this unit's check word (no-op otherwise)
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return (int)e;
    }
    // prefer the largest shared-memory carveout so that shared memory never
    // limits the blocks per SM below what registers allow
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    return (int)e;
}

// Streaming multiprocessors of the current device (queried once per device;
// grids of the grid-stride kernels are sized in multiples of it).
static inline int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

static inline size_t nd_of(const HostPlan &hp) { return hp.d == 2 ? (size_t)hp.N * hp.N : (size_t)hp.N * hp.N * hp.N; }
// points of f and Q (the N_in grid; the transform grid N is twice as fine
// in a de-aliased plan)
static inline size_t nd_in(const HostPlan &hp) {
    return hp.d == 2 ? (size_t)hp.N_in * hp.N_in : (size_t)hp.N_in * hp.N_in * hp.N_in;
}
static inline int cols_of(const HostPlan &hp) { return hp.d == 2 ? hp.N : hp.N * hp.N; }

// Warps of a line kernel that walks `lines` independent lines.
template <typename T, int N> static int line_warps(int lines) {
    return std::max(1, std::min(KCfg<T>::WARPS, lines / LineCfg<T, N>::LPW));
}

// Warps per block of a forward (FP64) line kernel over `lines` lines: the
// largest power of two up to KCfg::WARPS that keeps at least one block per SM
// and divides the lines, since FP64 line work is bound by each SM's FP64 units.
template <int N> static int spread_warps(int lines) {
    typedef FwdCfg<double, N> Cfg;   // the forward transform's line kernels
    int warps = 1;
    while (2 * warps <= KCfg<double>::WARPS && lines % (2 * warps * Cfg::LPW) == 0 &&
           lines / (2 * warps * Cfg::LPW) >= num_sms())
        warps *= 2;
    return warps;
}

// ------------------------------------------------------------------ forward
// Forward transform of f on its own grid (N = N_in).  A de-aliased plan
// writes the coefficients to ghat_in; the padding kernel moves them to the
// 2N grid.
// TC: the compute type of the forward transform (double; float on request
// for FP32 plans that are not de-aliased, with the plan's float twiddles).
template <typename T, int N, typename TC>
static int forward_nc(const HostPlan &hp, const DevicePtrs &p, cudaStream_t s) {
    typedef FwdCfg<TC, N> Cfg;
    const int P = hp.d == 2 ? N : N * N;
    cx<TC> *tmp = static_cast<cx<TC> *>(p.fwd_tmp);
    const cx<TC> *tw = sizeof(TC) == 8 ? reinterpret_cast<const cx<TC> *>(p.tw64) : static_cast<const cx<TC> *>(p.tw);
    int rc = 0;
    if (hp.d == 3) {
        if constexpr (N <= 64) {
            // rows (axis 2) of all N^2 rows, two real rows per transform, then
            // axes 1 and 0: line kernels over the whole grid, so every SM takes
            // part in the FP64 work
            const int rows = N * N / 2;
            const int warps = spread_warps<N>(rows);
            const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
            if ((rc = set_smem(k_fwd_rows_2d<T, N, TC, true>, smem))) return rc;
            k_fwd_rows_2d<T, N, TC, true><<<rows / (warps * Cfg::LPW), warps * 32, smem, s>>>(
                static_cast<const T *>(p.f), tmp, tw);
            // axes 1 and 0 over the Hermitian half j3 <= N/2 (f is real)
            const int half = N * (N / 2 + 1);
            const int hw = spread_warps<N>(half);
            const size_t hsmem = (size_t)(N + hw * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
            if ((rc = set_smem(k_fwd_mid_3d<N, TC>, hsmem))) return rc;
            k_fwd_mid_3d<N, TC><<<half / (hw * Cfg::LPW), hw * 32, hsmem, s>>>(tmp, tw);
            if ((rc = set_smem(k_fwd_cols<T, N, TC, true>, hsmem))) return rc;
            k_fwd_cols<T, N, TC, true><<<half / (hw * Cfg::LPW), hw * 32, hsmem, s>>>(
                tmp, static_cast<cx<T> *>(hp.dealias ? p.ghat_in : p.ghat), tw, P, hp.d, 1.0 / (double)nd_in(hp),
                hp.nyquist == WKE_NYQ_ZERO, hp.nyquist == WKE_NYQ_KEEP ? static_cast<cx<T> *>(p.nslice) : nullptr);
            return (int)cudaGetLastError();
        } else {
            return (int)cudaErrorInvalidValue;
        }
    } else {
        const int warps = spread_warps<N>(N);
        const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
        if ((rc = set_smem(k_fwd_rows_2d<T, N, TC>, smem))) return rc;
        k_fwd_rows_2d<T, N, TC><<<N / (warps * Cfg::LPW), warps * 32, smem, s>>>(static_cast<const T *>(p.f), tmp, tw);
    }
    const int warps = spread_warps<N>(P);
    const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
    if ((rc = set_smem(k_fwd_cols<T, N, TC>, smem))) return rc;
    const double inv_nd = 1.0 / (double)nd_in(hp);
    k_fwd_cols<T, N, TC><<<P / (warps * Cfg::LPW), warps * 32, smem, s>>>(
        tmp, static_cast<cx<T> *>(hp.dealias ? p.ghat_in : p.ghat), tw, P, hp.d, inv_nd, hp.nyquist == WKE_NYQ_ZERO,
        hp.nyquist == WKE_NYQ_KEEP ? static_cast<cx<T> *>(p.nslice) : nullptr);
    return (int)cudaGetLastError();
}

template <typename T, int N> static int forward_n(const HostPlan &hp, const DevicePtrs &p, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (hp.tune_forward_fp32 && !hp.dealias) return forward_nc<T, N, float>(hp, p, s);
    }
    return forward_nc<T, N, double>(hp, p, s);
}

// Q-hat of grid values Q (N_in grid, plan type T) into Qhat: the forward
// transform's three (two in 2D) line passes in double on the plan's forward
// scratch, normalised by N^-d, then the alternating sign of the grid offset.
template <typename T, int N>
static int spectrum_n(const HostPlan &hp, const DevicePtrs &p, const void *Q, void *Qhat, cudaStream_t s) {
    typedef double TC;
    typedef FwdCfg<TC, N> Cfg;
    const int P = hp.d == 2 ? N : N * N;
    cx<TC> *tmp = static_cast<cx<TC> *>(p.fwd_tmp);
    const cx<TC> *tw = reinterpret_cast<const cx<TC> *>(p.tw64);
    int rc = 0;
    if (hp.d == 3) {
        if constexpr (N <= 64) {
            // rows (axis 2) two real rows per transform
            const int rows = N * N / 2;
            const int warps = spread_warps<N>(rows);
            const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
            if ((rc = set_smem(k_fwd_rows_2d<T, N, TC, true>, smem))) return rc;
            k_fwd_rows_2d<T, N, TC, true><<<rows / (warps * Cfg::LPW), warps * 32, smem, s>>>(
                static_cast<const T *>(Q), tmp, tw);
            const int half = N * (N / 2 + 1);     // Hermitian half: Q is real
            const int hw = spread_warps<N>(half);
            const size_t hsmem = (size_t)(N + hw * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
            if ((rc = set_smem(k_fwd_mid_3d<N, TC>, hsmem))) return rc;
            k_fwd_mid_3d<N, TC><<<half / (hw * Cfg::LPW), hw * 32, hsmem, s>>>(tmp, tw);
        } else {
            return (int)cudaErrorInvalidValue;
        }
    } else {
        const int warps = spread_warps<N>(N);
        const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
        if ((rc = set_smem(k_fwd_rows_2d<T, N, TC>, smem))) return rc;
        k_fwd_rows_2d<T, N, TC><<<N / (warps * Cfg::LPW), warps * 32, smem, s>>>(static_cast<const T *>(Q), tmp, tw);
    }
    const size_t nd = (size_t)N * P;
    if (hp.d == 3) {
        if constexpr (N <= 64) {
            const int half = N * (N / 2 + 1);
            const int hw = spread_warps<N>(half);
            const size_t hsmem = (size_t)(N + hw * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
            if ((rc = set_smem(k_fwd_cols<T, N, TC, true>, hsmem))) return rc;
            k_fwd_cols<T, N, TC, true><<<half / (hw * Cfg::LPW), hw * 32, hsmem, s>>>(
                tmp, static_cast<cx<T> *>(Qhat), tw, P, hp.d, 1.0 / (double)nd, 0, nullptr);
        }
    } else {
        const int warps = spread_warps<N>(P);
        const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<TC>);
        if ((rc = set_smem(k_fwd_cols<T, N, TC>, smem))) return rc;
        k_fwd_cols<T, N, TC><<<P / (warps * Cfg::LPW), warps * 32, smem, s>>>(tmp, static_cast<cx<T> *>(Qhat), tw, P,
                                                                             hp.d, 1.0 / (double)nd, 0, nullptr);
    }
    const int blocks = (int)std::min<size_t>((nd + 255) / 256, (size_t)num_sms() * 8);
    k_alternate_sign<T><<<blocks, 256, 0, s>>>(static_cast<cx<T> *>(Qhat), hp.d, N, nd);
    return (int)cudaGetLastError();
}

template <typename T> int spectrum_T(const HostPlan &hp, const DevicePtrs &p, const void *Q, void *Qhat, cudaStream_t s) {
    switch (hp.N_in) {
        case 16: return spectrum_n<T, 16>(hp, p, Q, Qhat, s);
        case 32: return spectrum_n<T, 32>(hp, p, Q, Qhat, s);
        case 48: return spectrum_n<T, 48>(hp, p, Q, Qhat, s);
        case 64: return spectrum_n<T, 64>(hp, p, Q, Qhat, s);
        case 96: return spectrum_n<T, 96>(hp, p, Q, Qhat, s);
        case 128: return spectrum_n<T, 128>(hp, p, Q, Qhat, s);
        case 256: return spectrum_n<T, 256>(hp, p, Q, Qhat, s);
    }
    return (int)cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ pass 1
// Groups, fields and units of chunk c: per-group layout (g0, ng; sf0 = -1)
// or shared-field layout (fields sf0 .. sf0 + sK - 1).
struct ChunkRange {
    int g0, ng, sf0, sK, units;
};
static inline ChunkRange chunk_range(const HostPlan &hp, int c) {
    ChunkRange r;
    if (hp.shared) {
        r.g0 = hp.chunk_g0[c];
        r.ng = hp.chunk_g0[c + 1] - r.g0;
        r.sf0 = hp.chunk_f0[c];
        r.sK = hp.chunk_f0[c + 1] - r.sf0;
    } else {
        r.g0 = c * hp.groups_per_chunk;
        r.ng = std::min(hp.groups_per_chunk, hp.n_groups - r.g0);
        r.sf0 = -1;
        r.sK = 0;
    }
    r.units = units_of_chunk(hp, c);
    return r;
}

template <typename T, int N>
static int pass1_n(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef LineCfg<T, N> Cfg;
    const ChunkRange cr = chunk_range(hp, c);
    const int g0 = cr.g0, ng = cr.ng, nunits = cr.units;
    const cx<T> *ghat = static_cast<const cx<T> *>(p.ghat);
    const cx<T> *ph = static_cast<const cx<T> *>(p.phase);
    cx<T> *H = static_cast<cx<T> *>(p.H);
    const cx<T> *tw = static_cast<const cx<T> *>(p.tw);
    int rc = 0;
    if (hp.d == 3) {
        if constexpr (N <= 64) {
            const size_t smem = (size_t)(N + N * Work<N>::PITCH + N * LinePad<N>::PITCH + 8 * N + 4) * sizeof(cx<T>);
            if ((rc = set_smem(k_pass1_3d<T, N>, smem))) return rc;
            // enough blocks to fill the GPU several times over
            // automatic: 2 units per block in the shared-field layout (13-unit chunks
            // at 3D N=64 give 448 blocks), 3 in the per-group layout (18-unit chunks)
            const int upb = std::min(nunits, hp.tune_p1_units_per_block > 0 ? hp.tune_p1_units_per_block
                                                                            : (hp.shared ? 2 : 3));
            dim3 grid(N, (nunits + upb - 1) / upb);
            k_pass1_3d<T, N><<<grid, N * Cfg::TPL, smem, s>>>(ghat, ph, H, tw, p.prod_local, g0, ng,
                                                               hp.fields_per_group, hp.products_per_group, nunits, upb,
                                                               cr.sf0, cr.sK);
        } else {
            return (int)cudaErrorInvalidValue;
        }
    } else {
        const int warps = line_warps<T, N>(N);
        const size_t smem = (size_t)(N + warps * Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<T>);
        if ((rc = set_smem(k_pass1_2d<T, N>, smem))) return rc;
        dim3 grid(N / (warps * Cfg::LPW), nunits);
        k_pass1_2d<T, N><<<grid, warps * 32, smem, s>>>(ghat, ph, H, tw, p.prod_local, g0, ng, hp.fields_per_group,
                                                        hp.products_per_group, cr.sf0, cr.sK);
    }
    return (int)cudaGetLastError();
}

// Separable plans: the chunk's row values and pairs along axes 2 and 1 into S.
template <typename T, int N>
static int sep_planes_n(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef LineCfg<T, N> Cfg;
    if constexpr (N <= 64) {
        const int v0 = hp.chunk_v0[c], nv = hp.chunk_v0[c + 1] - v0;
        int rc = 0;
        if constexpr (N == 64 && sizeof(T) == 4) {       // warp-local lines
            int mvp = 0;    // most pairs of one row value: the staged E1 rows
            for (int v = v0; v < v0 + nv; ++v) mvp = std::max(mvp, hp.sep_v[3 * v + 2] - hp.sep_v[3 * v + 1]);
            const size_t smem64 = (size_t)(N + N * SepWork64<N>::WP + 16 * 256 + (1 + mvp) * N) * sizeof(float2);
            if ((rc = set_smem(k_sep_planes64<N>, smem64))) return rc;
            k_sep_planes64<N><<<dim3(N, nv), 512, smem64, s>>>(
                static_cast<const float2 *>(p.ghat), static_cast<const float2 *>(p.phase), static_cast<float2 *>(p.S),
                static_cast<const float2 *>(p.tw), p.sep_v, p.sep_p, v0, hp.chunk_p0[c], hp.n_fields_total,
                hp.max_chunk_pairs, mvp);
            return (int)cudaGetLastError();
        }
        const size_t smem = (size_t)(N + N * Work<N>::PITCH + N * LinePad<N>::PITCH) * sizeof(cx<T>);
        if ((rc = set_smem(k_sep_planes_3d<T, N>, smem))) return rc;
        k_sep_planes_3d<T, N><<<dim3(N, nv), N * Cfg::TPL, smem, s>>>(
            static_cast<const cx<T> *>(p.ghat), static_cast<const cx<T> *>(p.phase), static_cast<cx<T> *>(p.S),
            static_cast<const cx<T> *>(p.tw), p.sep_v, p.sep_p, v0, hp.chunk_p0[c]);
        return (int)cudaGetLastError();
    } else {
        return (int)cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ Nyquist tables
// Tables of every unit of chunk c, into p.V.
template <typename T, int N>
static int nyquist_n(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef LineCfg<T, N> Cfg;
    const ChunkRange cr = chunk_range(hp, c);
    const int upc = max_chunk_units(hp), chunk0 = hp.shared ? 0 : c, nchunks = 1;
    const cx<T> *ph = static_cast<const cx<T> *>(p.phase);
    cx<T> *V = static_cast<cx<T> *>(p.V);
    const cx<T> *tw = static_cast<const cx<T> *>(p.tw);
    const cx<T> *ns = static_cast<const cx<T> *>(p.nslice);
    int rc = 0;
    if (hp.d == 3) {
        if constexpr (N == 64 && sizeof(T) == 4) {       // warp-local lines
            // twiddles, rows, exchange slots, the staged slice, two fields' phase rows
            const size_t smem64 = (size_t)(N + 2 * N * SepWork64<N>::WP + 16 * 256 + 6 * N) * sizeof(float2);
            if ((rc = set_smem(k_nyquist64<N>, smem64))) return rc;
            k_nyquist64<N><<<dim3(3, upc, nchunks), 512, smem64, s>>>(
                reinterpret_cast<const float2 *>(ph), reinterpret_cast<float2 *>(V),
                reinterpret_cast<const float2 *>(tw), reinterpret_cast<const float2 *>(ns), p.prod_local,
                hp.groups_per_chunk, hp.n_groups, hp.fields_per_group, hp.products_per_group, upc, chunk0, cr.sf0,
                cr.sK);
            return (int)cudaGetLastError();
        }
        if constexpr (N <= 64) {
            const size_t smem = (size_t)(N + N * Work<N>::PITCH + N * LinePad<N>::PITCH) * sizeof(cx<T>);
            if ((rc = set_smem(k_nyquist_3d<T, N>, smem))) return rc;
            k_nyquist_3d<T, N><<<dim3(3, upc, nchunks), N * Cfg::TPL, smem, s>>>(
                ph, V, tw, ns, p.prod_local, hp.groups_per_chunk, hp.n_groups, hp.fields_per_group,
                hp.products_per_group, upc, chunk0, cr.sf0, cr.sK);
        } else {
            return (int)cudaErrorInvalidValue;
        }
    } else {
        const size_t smem = (size_t)(N + Cfg::LPW * LinePad<N>::PITCH) * sizeof(cx<T>);
        if ((rc = set_smem(k_nyquist_2d<T, N>, smem))) return rc;
        k_nyquist_2d<T, N><<<dim3((2 * upc + Cfg::LPW - 1) / Cfg::LPW, nchunks), 32, smem, s>>>(
            ph, V, tw, ns, p.prod_local, hp.groups_per_chunk, hp.n_groups, hp.fields_per_group,
            hp.products_per_group, upc, chunk0, cr.sf0, cr.sK);
    }
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ shared-field layout
template <typename T, int N, int EP> static int axis0_ne(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef Pass2Cfg<T, N, EP> Cfg;
    const int P = cols_of(hp);
    int CB = std::min(Cfg::CB, P);
    while (P % CB) CB /= 2;
    const size_t smem = (size_t)(N + LinePad<N>::LEN * CB) * sizeof(cx<T>);
    int rc = 0;
    if ((rc = set_smem(k_axis0<T, N, EP>, smem))) return rc;
    k_axis0<T, N, EP><<<dim3(P / CB, units_of_chunk(hp, c)), CB * Cfg::TPL, smem, s>>>(
        static_cast<cx<T> *>(p.H), static_cast<const cx<T> *>(p.tw), P, CB);
    return (int)cudaGetLastError();
}

template <typename T, int N, int EP>
static int axis0_sep_ne(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef Pass2Cfg<T, N, EP> Cfg;
    const ChunkRange cr = chunk_range(hp, c);
    const int P = cols_of(hp);
    int CB = std::min(Cfg::CB, P);
    while (P % CB) CB /= 2;
    const size_t smem = (size_t)(N + LinePad<N>::LEN * CB) * sizeof(cx<T>);
    int rc = 0;
    if ((rc = set_smem(k_axis0_sep<T, N, EP>, smem))) return rc;
    k_axis0_sep<T, N, EP><<<dim3(P / CB, cr.units), CB * Cfg::TPL, smem, s>>>(
        static_cast<const cx<T> *>(p.S), static_cast<const cx<T> *>(p.phase), p.field_pair, static_cast<cx<T> *>(p.H),
        static_cast<const cx<T> *>(p.tw), P, CB, cr.sf0, cr.sK, hp.max_chunk_pairs);
    return (int)cudaGetLastError();
}

template <typename T, int N> static int axis0_n(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    if (hp.separable) {
        if constexpr (N % 3 == 0) {
            return axis0_sep_ne<T, N, 12>(hp, p, c, s);
        } else {
            if constexpr (N <= 64) {
                if (hp.tune_p2_points == 8) return axis0_sep_ne<T, N, 8>(hp, p, c, s);
            }
            return axis0_sep_ne<T, N, 4>(hp, p, c, s);
        }
    }
    if constexpr (N % 3 == 0) {
        return axis0_ne<T, N, 12>(hp, p, c, s);
    } else {
        if constexpr (N <= 64) {
            if (hp.tune_p2_points == 8) return axis0_ne<T, N, 8>(hp, p, c, s);
        }
        return axis0_ne<T, N, 4>(hp, p, c, s);
    }
}

// ------------------------------------------------------------------ fused axis 0 + products
template <typename T, int N, bool SEP, bool IM, bool NYQ, int PPGC>
static int fused_nimp(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    typedef LineCfg<T, N> Cfg;
    constexpr int CB = Cfg::LPW, PTS = N * CB;
    const ChunkRange cr = chunk_range(hp, c);
    FusedTab<T> tab;
    const int np = cr.ng * hp.products_per_group;
    if (np > FusedTab<T>::kMaxProducts || cr.ng > FusedTab<T>::kMaxGroups || cr.sK > 255)
        return (int)cudaErrorInvalidValue;
    for (int i = 0; i < np; ++i) {
        const int slot = cr.g0 * hp.products_per_group + i;
        tab.pa[i] = (unsigned char)hp.prod_fa[slot];
        tab.pb[i] = (unsigned char)hp.prod_fb[slot];
        tab.w[i] = (T)hp.prod_W[slot];
    }
    for (int g = 0; g < cr.ng; ++g) tab.cf[g] = (unsigned char)hp.group_cfield[cr.g0 + g];
    if constexpr (N == 64 && sizeof(T) == 4) {
        // field slots, staged planes and twiddles, when they fit
        const int U = (cr.sK + 1) / 2;
        const int nplanes = SEP ? hp.chunk_p0[c + 1] - hp.chunk_p0[c] : U;
        const size_t smem64 = ((size_t)(2 * U + nplanes) * kF64Pts + N) * sizeof(float2);
        if (smem64 <= kMaxDynamicSmem && U <= Fused64Tab::kMaxUnits) {
            Fused64Tab t64;
            // byte offset of a chunk-local field from its point's unit entry:
            // the two fields of unit u are interleaved (k_fused64)
            auto foff = [](int l) { return (unsigned)((l >> 1) * kF64Pts * sizeof(float4) + (l & 1) * sizeof(float2)); };
            for (int i = 0; i < np; ++i) {
                t64.oa[i] = foff(tab.pa[i]);
                t64.ob[i] = foff(tab.pb[i]);
                t64.w[i] = (float)tab.w[i];
            }
            for (int g = 0; g < cr.ng; ++g) t64.oc[g] = foff(tab.cf[g]);
            if (SEP)
                for (int u = 0; u < U; ++u) {
                    const int fa = cr.sf0 + 2 * u, fb = 2 * u + 1 < cr.sK ? fa + 1 : fa;
                    t64.pla[u] = (unsigned char)hp.field_pair[fa];
                    t64.plb[u] = (unsigned char)hp.field_pair[fb];
                }
            const int ubase = hp.chunk_u0[c];
            // one weight per group (every equal-weight sphere rule): the factored product sum
            bool eqw = PPGC > 0;
            for (int g = 0; g < cr.ng && eqw; ++g)
                for (int q = 1; q < PPGC; ++q) eqw = eqw && t64.w[g * PPGC + q] == t64.w[g * PPGC];
            int rc = 0;
#define WKE_F64_LAUNCH(NGC_, EQW_, CUBE_)                                                                       \
    do {                                                                                                        \
        if ((rc = set_smem(k_fused64<SEP, IM, NYQ, PPGC, NGC_, EQW_, CUBE_>, smem64))) return rc;                \
        k_fused64<SEP, IM, NYQ, PPGC, NGC_, EQW_, CUBE_><<<(N * N) / 4, kF64Pts, smem64, s>>>(                   \
            static_cast<const float2 *>(SEP ? p.S : p.H), static_cast<const float4 *>(p.unit_e0),                 \
            static_cast<const float2 *>(p.V), static_cast<const float *>(p.f), p.Qacc, p.Qacc_im,                \
            static_cast<const float2 *>(p.tw), cr.sK, cr.ng, hp.products_per_group, nplanes, ubase, t64,          \
            static_cast<float *>(p.Qout), static_cast<float *>(p.Qiout), p.scale_out);                          \
    } while (0)
            if constexpr (PPGC == 3) {
                const HostPlan::CubeChunk *cu = hp.cube.empty() ? nullptr : &hp.cube[c];
                // the kernel reads the fields in the order the plan gives them
                // (edges, faces, C fields; wke_plan.cpp, order_cube_fields)
                bool canonical = cu != nullptr && cr.sK == 26;
                for (int i = 0; i < 6 && canonical; ++i) canonical = cu->edge[i] == i;
                for (int i = 0; i < 12 && canonical; ++i) canonical = cu->face[i] == 6 + i;
                for (int v = 0; v < 8 && canonical; ++v) canonical = cu->cfield[v] == 18 + v;
                if (canonical && hp.tune_rule_products) {
                    // the cube rule's schedule: every field read once per point
                    for (int v = 0; v < 8; ++v) t64.w[v] = (float)cu->w[v];
                    WKE_F64_LAUNCH(8, true, true);
                    return (int)cudaGetLastError();
                }
            }
            if constexpr (PPGC == 3 || PPGC == 4) {
                if (cr.ng == 8 && eqw) WKE_F64_LAUNCH(8, true, false);
                else if (cr.ng == 8) WKE_F64_LAUNCH(8, false, false);
                else WKE_F64_LAUNCH(0, false, false);
            } else {
                WKE_F64_LAUNCH(0, false, false);
            }
#undef WKE_F64_LAUNCH
            return (int)cudaGetLastError();
        }
    }
    const size_t smem = fused_smem_bytes(N, cr.sK);
    int rc = 0;
    if ((rc = set_smem(k_fused_3d<T, N, SEP, IM, NYQ, PPGC>, smem))) return rc;
    k_fused_3d<T, N, SEP, IM, NYQ, PPGC><<<(N * N) / CB, PTS, smem, s>>>(
        static_cast<const cx<T> *>(SEP ? p.S : p.H), static_cast<const cx<T> *>(p.phase), p.field_pair,
        static_cast<const cx<T> *>(p.V), static_cast<const T *>(p.f), p.Qacc, p.Qacc_im,
        static_cast<const cx<T> *>(p.tw), cr.sf0, cr.sK, cr.ng, hp.products_per_group, tab, static_cast<T *>(p.Qout),
        static_cast<T *>(p.Qiout), p.scale_out);
    return (int)cudaGetLastError();
}

template <typename T, int N, bool SEP, bool IM, bool NYQ>
static int fused_nim(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    switch (hp.products_per_group) {
    case 1: return fused_nimp<T, N, SEP, IM, NYQ, 1>(hp, p, c, s);
    case 2: return fused_nimp<T, N, SEP, IM, NYQ, 2>(hp, p, c, s);
    case 3: return fused_nimp<T, N, SEP, IM, NYQ, 3>(hp, p, c, s);
    case 4: return fused_nimp<T, N, SEP, IM, NYQ, 4>(hp, p, c, s);
    default: return fused_nimp<T, N, SEP, IM, NYQ, 0>(hp, p, c, s);
    }
}

template <typename T, int N, bool SEP>
static int fused_ns(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    const bool nyq = hp.nyquist == WKE_NYQ_KEEP;
    if (nyq) return im ? fused_nim<T, N, SEP, true, true>(hp, p, c, s) : fused_nim<T, N, SEP, false, true>(hp, p, c, s);
    return im ? fused_nim<T, N, SEP, true, false>(hp, p, c, s) : fused_nim<T, N, SEP, false, false>(hp, p, c, s);
}

// Instantiated in translation units of their own (wke_fused*.cu), which keeps
// each compilation short; the other units see them as extern templates.
template <typename T, int N>
int fused_at(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && N <= 64) {
        return hp.separable ? fused_ns<T, N, true>(hp, p, c, im, s) : fused_ns<T, N, false>(hp, p, c, im, s);
    } else {
        return (int)cudaErrorInvalidValue;
    }
}

template <typename T, bool IM, bool NYQ, int PPGC>
static int products_nimp(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    const ChunkRange cr = chunk_range(hp, c);
    const int P = cols_of(hp);
    const size_t ND = nd_of(hp);
    if (P % kProductThreads == 0) {
        // staged kernel (3D, and 2D rows of at least a block), when its shared memory fits
        const int U = (cr.sK + 1) / 2;
        int W2 = 0, TS = 2;                   // 2D: one V_1 entry per unit (two keep 16-byte alignment)
        if (hp.d == 3) {
            W2 = kProductThreads / hp.N + 2;  // V_2 entries a block's columns use, at most
            W2 += (hp.N + W2) & 1;            // keeps each unit's table 16-byte aligned
            TS = hp.N + W2;
        }
        const size_t smem3 = ((size_t)2 * U * kProductThreads + (NYQ ? (size_t)U * TS : 0)) * sizeof(cx<T>) +
                             (size_t)cr.ng * hp.products_per_group * sizeof(ProdEntry<T>) + (size_t)cr.ng * sizeof(int);
        if (smem3 <= kMaxDynamicSmem) {
            int rc = 0;
            if ((rc = set_smem(k_products_staged<T, IM, NYQ, PPGC>, smem3))) return rc;
            k_products_staged<T, IM, NYQ, PPGC><<<(unsigned)(ND / kProductThreads), kProductThreads, smem3, s>>>(
                static_cast<const cx<T> *>(p.H), static_cast<const cx<T> *>(p.V), static_cast<const T *>(p.f), p.Qacc,
                p.Qacc_im, p.group_cfield, p.prod_local, p.prod_W, hp.d, hp.N, P, cr.g0, cr.ng, cr.sK,
                hp.products_per_group, TS, W2);
            return (int)cudaGetLastError();
        }
    }
    const size_t smem = (size_t)cr.sK * kProductThreads * sizeof(cx<T>) +
                        (size_t)cr.ng * hp.products_per_group * sizeof(ProdEntry<T>) + (size_t)cr.ng * sizeof(int);
    int rc = 0;
    if ((rc = set_smem(k_products<T, IM, NYQ, PPGC>, smem))) return rc;
    const int blocks = (int)std::min<size_t>((ND + kProductThreads - 1) / kProductThreads, num_sms() * 16);
    k_products<T, IM, NYQ, PPGC><<<blocks, kProductThreads, smem, s>>>(
        static_cast<const cx<T> *>(p.H), static_cast<const cx<T> *>(p.V), static_cast<const T *>(p.f), p.Qacc,
        p.Qacc_im, p.group_cfield, p.prod_local, p.prod_W, hp.d, hp.N, P, cr.g0, cr.ng, cr.sK,
        hp.products_per_group);
    return (int)cudaGetLastError();
}

// The product count per group is a template constant for the counts the
// built-in rules give (1 to 4), so that the product loop unrolls.
template <typename T, bool IM, bool NYQ>
static int products_nim(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    switch (hp.products_per_group) {
    case 1: return products_nimp<T, IM, NYQ, 1>(hp, p, c, s);
    case 2: return products_nimp<T, IM, NYQ, 2>(hp, p, c, s);
    case 3: return products_nimp<T, IM, NYQ, 3>(hp, p, c, s);
    case 4: return products_nimp<T, IM, NYQ, 4>(hp, p, c, s);
    default: return products_nimp<T, IM, NYQ, 0>(hp, p, c, s);
    }
}

template <typename T>
int products_T(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    const bool nyq = hp.nyquist == WKE_NYQ_KEEP;
    if (nyq) return im ? products_nim<T, true, true>(hp, p, c, s) : products_nim<T, false, true>(hp, p, c, s);
    return im ? products_nim<T, true, false>(hp, p, c, s) : products_nim<T, false, false>(hp, p, c, s);
}

// ------------------------------------------------------------------ pass 2
template <typename T, int N, int EP, bool IM, bool NYQ>
static int pass2_nim(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    const ChunkRange cr = chunk_range(hp, c);
    const int g0 = cr.g0, ng = cr.ng;
    typedef Pass2Cfg<T, N, EP> Cfg;
    const int P = cols_of(hp);
    int CB = std::min(Cfg::CB, P);             // columns per block: a power of two dividing P
    while (P % CB) CB /= 2;
    // two stage buffers for unit tiles, and with the Nyquist set kept in 3D
    // three slots of staged table entries
    const size_t vslots = NYQ && hp.d == 3 && N % CB == 0 ? (size_t)3 * (N * CB + N + CB) : 0;
    const size_t smem = (size_t)(N + LinePad<N>::LEN * CB + 2 * N * CB + vslots) * sizeof(cx<T>);
    int rc = 0;
    if ((rc = set_smem(k_pass2<T, N, EP, IM, NYQ>, smem))) return rc;
    dim3 grid(P / CB, ng);
    k_pass2<T, N, EP, IM, NYQ><<<grid, CB * Cfg::TPL, smem, s>>>(
        static_cast<const cx<T> *>(p.H), static_cast<const cx<T> *>(p.V), static_cast<const T *>(p.f), p.Qacc,
        p.Qacc_im, p.prod_local, p.prod_W, static_cast<const cx<T> *>(p.tw), hp.d, P, CB, hp.products_per_group, g0,
        ng);
    return (int)cudaGetLastError();
}

template <typename T, int N, int EP>
static int pass2_ne(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    const bool nyq = hp.nyquist == WKE_NYQ_KEEP;
    if (nyq)
        return im ? pass2_nim<T, N, EP, true, true>(hp, p, c, s) : pass2_nim<T, N, EP, false, true>(hp, p, c, s);
    return im ? pass2_nim<T, N, EP, true, false>(hp, p, c, s) : pass2_nim<T, N, EP, false, false>(hp, p, c, s);
}

template <typename T, int N>
static int pass2_n(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    if constexpr (N % 3 == 0) {
        return pass2_ne<T, N, 12>(hp, p, c, im, s);
    } else {
        if constexpr (N <= 64) {
            if (hp.tune_p2_points == 8) return pass2_ne<T, N, 8>(hp, p, c, im, s);
        }
        return pass2_ne<T, N, 4>(hp, p, c, im, s);
    }
}

// ------------------------------------------------------------------ dispatch on N
template <typename T> int forward_T(const HostPlan &hp, const DevicePtrs &p, cudaStream_t s) {
    switch (hp.N_in) {
        case 16: return forward_n<T, 16>(hp, p, s);
        case 32: return forward_n<T, 32>(hp, p, s);
        case 48: return forward_n<T, 48>(hp, p, s);
        case 64: return forward_n<T, 64>(hp, p, s);
        case 96: return forward_n<T, 96>(hp, p, s);
        case 128: return forward_n<T, 128>(hp, p, s);
        case 256: return forward_n<T, 256>(hp, p, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T> int pass1_T(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    switch (hp.N) {
        case 16: return pass1_n<T, 16>(hp, p, c, s);
        case 32: return pass1_n<T, 32>(hp, p, c, s);
        case 48: return pass1_n<T, 48>(hp, p, c, s);
        case 64: return pass1_n<T, 64>(hp, p, c, s);
        case 96: return pass1_n<T, 96>(hp, p, c, s);
        case 128: return pass1_n<T, 128>(hp, p, c, s);
        case 256: return pass1_n<T, 256>(hp, p, c, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T> int nyquist_T(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    switch (hp.N) {
        case 16: return nyquist_n<T, 16>(hp, p, c, s);
        case 32: return nyquist_n<T, 32>(hp, p, c, s);
        case 48: return nyquist_n<T, 48>(hp, p, c, s);
        case 64: return nyquist_n<T, 64>(hp, p, c, s);
        case 96: return nyquist_n<T, 96>(hp, p, c, s);
        case 128: return nyquist_n<T, 128>(hp, p, c, s);
        case 256: return nyquist_n<T, 256>(hp, p, c, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T>
int pass2_T(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    switch (hp.N) {
        case 16: return pass2_n<T, 16>(hp, p, c, im, s);
        case 32: return pass2_n<T, 32>(hp, p, c, im, s);
        case 48: return pass2_n<T, 48>(hp, p, c, im, s);
        case 64: return pass2_n<T, 64>(hp, p, c, im, s);
        case 96: return pass2_n<T, 96>(hp, p, c, im, s);
        case 128: return pass2_n<T, 128>(hp, p, c, im, s);
        case 256: return pass2_n<T, 256>(hp, p, c, im, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <int N> static int axis0_tc_n(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    const int P = cols_of(hp);
    k_axis0_tc<N><<<dim3(P / 32, units_of_chunk(hp, c)), N / 16 * 32, 0, s>>>(
        static_cast<float2 *>(p.H), static_cast<const float2 *>(p.tw), P);
    return (int)cudaGetLastError();
}

template <typename T> int axis0_T(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (hp.split) {
            if (hp.N == 64) return axis0_tc_n<64>(hp, p, c, s);
            if (hp.N == 32) return axis0_tc_n<32>(hp, p, c, s);
            return (int)cudaErrorInvalidValue;
        }
    }
    switch (hp.N) {
        case 16: return axis0_n<T, 16>(hp, p, c, s);
        case 32: return axis0_n<T, 32>(hp, p, c, s);
        case 48: return axis0_n<T, 48>(hp, p, c, s);
        case 64: return axis0_n<T, 64>(hp, p, c, s);
        case 96: return axis0_n<T, 96>(hp, p, c, s);
        case 128: return axis0_n<T, 128>(hp, p, c, s);
        case 256: return axis0_n<T, 256>(hp, p, c, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T> int sep_planes_T(const HostPlan &hp, const DevicePtrs &p, int c, cudaStream_t s) {
    switch (hp.N) {
        case 16: return sep_planes_n<T, 16>(hp, p, c, s);
        case 32: return sep_planes_n<T, 32>(hp, p, c, s);
        case 48: return sep_planes_n<T, 48>(hp, p, c, s);
        case 64: return sep_planes_n<T, 64>(hp, p, c, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T> int fused_T(const HostPlan &hp, const DevicePtrs &p, int c, bool im, cudaStream_t s) {
    switch (hp.N) {
        case 16: return fused_at<T, 16>(hp, p, c, im, s);
        case 32: return fused_at<T, 32>(hp, p, c, im, s);
        case 48: return fused_at<T, 48>(hp, p, c, im, s);
        case 64: return fused_at<T, 64>(hp, p, c, im, s);
    }
    return (int)cudaErrorInvalidValue;
}

template <typename T>
int finalize_T(const HostPlan &hp, const DevicePtrs &p, void *Q, void *Qim, cudaStream_t s) {
    const size_t ND = nd_of(hp);
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((ND + threads - 1) / threads, num_sms() * 8);
    k_finalize<T><<<blocks, threads, 0, s>>>(p.Qacc, Qim ? p.Qacc_im : nullptr, n_accumulators(hp), ND, hp.scale,
                                             static_cast<T *>(Q), static_cast<T *>(Qim));
    return (int)cudaGetLastError();
}

template <typename T>
int moments_T(const HostPlan &hp, const void *g, double *partials, double *out, cudaStream_t s) {
    k_moments<T><<<kMomentBlocks, kMomentThreads, 0, s>>>(static_cast<const T *>(g), hp.d, hp.N_in, hp.L, partials);
    const double h = 2.0 * hp.L / hp.N_in;
    const double hd = hp.d == 2 ? h * h : h * h * h;
    k_moments_reduce<<<1, 32, 0, s>>>(partials, kMomentBlocks, hp.d + 2, hd, out);
    return (int)cudaGetLastError();
}

template <typename T>
int rk_stage_T(const HostPlan &hp, const void *f, const void *k, double *kacc, void *ystage, double b_s,
               double c_next_dt, int first, cudaStream_t s) {
    const size_t ND = nd_in(hp);
    const int blocks = (int)std::min<size_t>((ND + 255) / 256, num_sms() * 8);
    k_rk_stage<T><<<blocks, 256, 0, s>>>(static_cast<const T *>(f), static_cast<const T *>(k), kacc,
                                          static_cast<T *>(ystage), b_s, c_next_dt, first, ND);
    return (int)cudaGetLastError();
}

template <typename T> int rk_final_T(const HostPlan &hp, void *f, const double *kacc, double dt, cudaStream_t s) {
    const size_t ND = nd_in(hp);
    const int blocks = (int)std::min<size_t>((ND + 255) / 256, num_sms() * 8);
    k_rk_final<T><<<blocks, 256, 0, s>>>(static_cast<T *>(f), kacc, dt, ND);
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ de-aliasing
// One axis map per call: `in` viewed as [A][n_in][B], `out` as [A][n_out][B].
template <typename TIn, typename TOut>
static int axis_map(const TIn *in, TOut *out, TOut *out_im, const double2 *K, int n_out, int n_in, size_t A, size_t B,
                    cudaStream_t s) {
    const size_t total = A * (size_t)n_out * B;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, num_sms() * 16);
    k_axis_map<TIn, TOut><<<blocks, 256, 0, s>>>(in, out, out_im, K, n_out, n_in, A, B);
    return (int)cudaGetLastError();
}

// Before the chunks: the coefficients on the 2N grid (padding) and
// F = f_N on the 2N grid, by the per-axis interpolation map applied to f.
template <typename T> int dealias_prepare_T(const HostPlan &hp, const DevicePtrs &p, cudaStream_t s) {
    const size_t ND = nd_of(hp);
    const int blocks = (int)std::min<size_t>((ND + 255) / 256, num_sms() * 8);
    k_pad_spectrum<T><<<blocks, 256, 0, s>>>(static_cast<const cx<T> *>(p.ghat_in), static_cast<cx<T> *>(p.ghat), hp.d,
                                             hp.N_in, hp.N, ND);
    int rc = (int)cudaGetLastError();
    const int n = hp.N, m = hp.N_in;
    const double2 *K = static_cast<const double2 *>(p.Kint);
    double2 *b0 = static_cast<double2 *>(p.map0), *b1 = static_cast<double2 *>(p.map1);
    const T *f = static_cast<const T *>(p.f);
    T *ff = static_cast<T *>(p.ffine);
    if (hp.d == 2) {
        if (!rc) rc = axis_map<T, double2>(f, b0, nullptr, K, n, m, 1, m, s);
        if (!rc) rc = axis_map<double2, T>(b0, ff, nullptr, K, n, m, n, 1, s);
    } else {
        if (!rc) rc = axis_map<T, double2>(f, b0, nullptr, K, n, m, 1, (size_t)m * m, s);
        if (!rc) rc = axis_map<double2, double2>(b0, b1, nullptr, K, n, m, n, m, s);
        if (!rc) rc = axis_map<double2, T>(b1, ff, nullptr, K, n, m, (size_t)n * n, 1, s);
    }
    return rc;
}

// After the chunks: the weighted sum on the 2N grid (scaled, real: the
// padded fields of a Nyquist-zeroed f are real) projected onto the modes
// [-N_in/2, N_in/2-1]^d of the N_in grid; real part to Q, imaginary part
// (from the unpaired -N_in/2 modes of the projection) to Qim.
template <typename T> int dealias_finish_T(const HostPlan &hp, const DevicePtrs &p, void *Q, void *Qim, cudaStream_t s) {
    const size_t ND = nd_of(hp);
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((ND + threads - 1) / threads, num_sms() * 8);
    double *qf = static_cast<double *>(p.map0);
    if (hp.fused)   // FP32 fused layouts accumulate in (hi, lo) float pairs
        k_finalize_pair<double><<<blocks, threads, 0, s>>>(p.Qacc, ND, hp.scale, qf);
    else
        k_finalize<double><<<blocks, threads, 0, s>>>(p.Qacc, nullptr, n_accumulators(hp), ND, hp.scale, qf, nullptr);
    int rc = (int)cudaGetLastError();
    const int n = hp.N, m = hp.N_in;
    const double2 *K = static_cast<const double2 *>(p.Kproj);
    double2 *b0 = static_cast<double2 *>(p.map0), *b1 = static_cast<double2 *>(p.map1);
    T *q = static_cast<T *>(Q), *qi = static_cast<T *>(Qim);
    if (hp.d == 2) {
        if (!rc) rc = axis_map<double, double2>(qf, b1, nullptr, K, m, n, 1, n, s);
        if (!rc) rc = axis_map<double2, T>(b1, q, qi, K, m, n, m, 1, s);
    } else {
        if (!rc) rc = axis_map<double, double2>(qf, b1, nullptr, K, m, n, 1, (size_t)n * n, s);
        if (!rc) rc = axis_map<double2, double2>(b1, b0, nullptr, K, m, n, m, n, s);
        if (!rc) rc = axis_map<double2, T>(b0, q, qi, K, m, n, (size_t)m * m, 1, s);
    }
    return rc;
}

#define WKE_FUSED_AT(T, N) int fused_at<T, N>(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);
#define WKE_EXTERN_FUSED(T)                                                                                  \
    extern template WKE_FUSED_AT(T, 16) extern template WKE_FUSED_AT(T, 32) extern template WKE_FUSED_AT(T, 48) \
    extern template WKE_FUSED_AT(T, 64)

#define WKE_INSTANTIATE(T)                                                                                   \
    template int dealias_prepare_T<T>(const HostPlan &, const DevicePtrs &, cudaStream_t);                 \
    template int dealias_finish_T<T>(const HostPlan &, const DevicePtrs &, void *, void *, cudaStream_t);  \
    template int forward_T<T>(const HostPlan &, const DevicePtrs &, cudaStream_t);                         \
    template int spectrum_T<T>(const HostPlan &, const DevicePtrs &, const void *, void *, cudaStream_t);  \
    template int pass1_T<T>(const HostPlan &, const DevicePtrs &, int, cudaStream_t);                      \
    template int nyquist_T<T>(const HostPlan &, const DevicePtrs &, int, cudaStream_t);                    \
    template int pass2_T<T>(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);                \
    template int axis0_T<T>(const HostPlan &, const DevicePtrs &, int, cudaStream_t);                      \
    template int products_T<T>(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);             \
    template int sep_planes_T<T>(const HostPlan &, const DevicePtrs &, int, cudaStream_t);                 \
    template int fused_T<T>(const HostPlan &, const DevicePtrs &, int, bool, cudaStream_t);                \
    template int finalize_T<T>(const HostPlan &, const DevicePtrs &, void *, void *, cudaStream_t);        \
    template int moments_T<T>(const HostPlan &, const void *, double *, double *, cudaStream_t);           \
    template int rk_stage_T<T>(const HostPlan &, const void *, const void *, double *, void *, double,     \
                               double, int, cudaStream_t);                                                  \
    template int rk_final_T<T>(const HostPlan &, void *, const double *, double, cudaStream_t);

}  // namespace wke
