// Device building blocks: complex arithmetic, radix-2/3/4/8/12/16 DFTs in
// registers, and a warp-local Stockham line transform.
//
// Line transform layout.  A line of N points is held by TPL = N / E threads
// of one warp, E points each: thread t holds x[t + e * TPL] in v[e] on entry
// and X[t + e * TPL] in v[e] on exit (the Stockham autosort order keeps this
// distribution).  A warp holds LPW = 32 / TPL lines; lane = c + LPW * t for
// line c of the warp.  Between radix stages the points move through a
// per-line shared-memory scratch, padded by one slot per 8 so that the
// strided stage writes fall into distinct banks; only __syncwarp is needed.
//
// Lengths are 2^a (radix-8 or radix-4 stages, then a shorter one) or 3 * 2^a
// (a radix-12 stage first, then powers of two).
// Stage s of radix R after radices with product Ns handles butterflies
// j = t + u * TPL (u < E / R) on inputs x[j + r N / R], twiddles them by
// w_N^{(j mod Ns) r N / (Ns R)}, applies the R-point DFT and writes output r
// to position (j / Ns) Ns R + (j mod Ns) + r Ns.  DIR = +1 is the inverse
// transform (exp(+2 pi i nk/N), unnormalised), DIR = -1 the forward one.
#pragma once

#include <cuda_runtime.h>

namespace wke {

template <typename T> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };
template <typename T> using cx = typename CxT<T>::type;

template <typename T> __device__ __forceinline__ cx<T> mkc(T x, T y) {
    cx<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// FP32: the two lanes of a complex sum in one packed f32x2 instruction
// (each lane rounded as a scalar add).
__device__ __forceinline__ unsigned long long pack2(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
template <> __device__ __forceinline__ float2 cadd<float>(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
template <> __device__ __forceinline__ float2 csub<float>(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
// multiply by DIR * i
template <typename T, int DIR> __device__ __forceinline__ cx<T> mul_i(cx<T> a) {
    return DIR > 0 ? mkc<T>(-a.y, a.x) : mkc<T>(a.y, -a.x);
}
// multiply by (c + DIR * i * s)
template <typename T, int DIR> __device__ __forceinline__ cx<T> mul_cs(cx<T> a, T c, T s) {
    const T sd = DIR > 0 ? s : -s;
    return mkc<T>(a.x * c - a.y * sd, a.x * sd + a.y * c);
}

// ------------------------------------------------------------ small DFTs
// In place, natural order in and out: a[k] <- sum_n a[n] exp(DIR 2 pi i nk/R).
template <typename T, int R, int DIR> struct Dft;

template <typename T, int DIR> struct Dft<T, 2, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        cx<T> t = a[0];
        a[0] = cadd<T>(t, a[1]);
        a[1] = csub<T>(t, a[1]);
    }
};

template <typename T, int DIR> struct Dft<T, 4, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        cx<T> t0 = cadd<T>(a[0], a[2]), t1 = csub<T>(a[0], a[2]);
        cx<T> t2 = cadd<T>(a[1], a[3]), t3 = mul_i<T, DIR>(csub<T>(a[1], a[3]));
        a[0] = cadd<T>(t0, t2);
        a[2] = csub<T>(t0, t2);
        a[1] = cadd<T>(t1, t3);
        a[3] = csub<T>(t1, t3);
    }
};

// 3: X0 = a0 + (a1 + a2), X1,2 = a0 - (a1 + a2) / 2 +- DIR i (sqrt(3) / 2) (a1 - a2).
template <typename T, int DIR> struct Dft<T, 3, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        const T r3 = (T)0.86602540378443864676;   // sqrt(3) / 2
        const cx<T> s = cadd<T>(a[1], a[2]);
        const cx<T> dd = mul_i<T, DIR>(cscale<T>(csub<T>(a[1], a[2]), r3));
        const cx<T> m = csub<T>(a[0], cscale<T>(s, (T)0.5));
        a[0] = cadd<T>(a[0], s);
        a[1] = cadd<T>(m, dd);
        a[2] = csub<T>(m, dd);
    }
};

// 8 = 2 x 4: DFT4 of the even and odd samples, twiddle, radix-2 combine.
template <typename T, int DIR> struct Dft<T, 8, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        const T h = (T)0.70710678118654752440;   // 1/sqrt(2)
        cx<T> e[4] = {a[0], a[2], a[4], a[6]};
        cx<T> o[4] = {a[1], a[3], a[5], a[7]};
        Dft<T, 4, DIR>::run(e);
        Dft<T, 4, DIR>::run(o);
        o[1] = mul_cs<T, DIR>(o[1], h, h);
        o[2] = mul_i<T, DIR>(o[2]);
        o[3] = mul_cs<T, DIR>(o[3], -h, h);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = cadd<T>(e[k], o[k]);
            a[k + 4] = csub<T>(e[k], o[k]);
        }
    }
};

// 16 = 4 x 4: X[k1 + 4 k2] = sum_{n2} w16^{n2 k1} w4^{n2 k2} sum_{n1} a[4 n1 + n2] w4^{n1 k1}.
template <typename T, int DIR> struct Dft<T, 16, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        const T c1 = (T)0.92387953251128675613;   // cos(pi/8)
        const T s1 = (T)0.38268343236508977173;   // sin(pi/8)
        const T h = (T)0.70710678118654752440;
        cx<T> b[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            b[n2][0] = a[n2];
            b[n2][1] = a[4 + n2];
            b[n2][2] = a[8 + n2];
            b[n2][3] = a[12 + n2];
            Dft<T, 4, DIR>::run(b[n2]);
        }
        // twiddles w16^{n2 k1}, n2, k1 in 1..3
        b[1][1] = mul_cs<T, DIR>(b[1][1], c1, s1);
        b[1][2] = mul_cs<T, DIR>(b[1][2], h, h);
        b[1][3] = mul_cs<T, DIR>(b[1][3], s1, c1);
        b[2][1] = mul_cs<T, DIR>(b[2][1], h, h);
        b[2][2] = mul_i<T, DIR>(b[2][2]);
        b[2][3] = mul_cs<T, DIR>(b[2][3], -h, h);
        b[3][1] = mul_cs<T, DIR>(b[3][1], s1, c1);
        b[3][2] = mul_cs<T, DIR>(b[3][2], -h, h);
        b[3][3] = mul_cs<T, DIR>(b[3][3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cx<T> c[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
            Dft<T, 4, DIR>::run(c);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = c[k2];
        }
    }
};

// 12 = 3 x 4: X[k1 + 3 k2] = sum_{n2} w12^{n2 k1} w4^{n2 k2} sum_{n1} a[4 n1 + n2] w3^{n1 k1}.
template <typename T, int DIR> struct Dft<T, 12, DIR> {
    __device__ __forceinline__ static void run(cx<T> *a) {
        const T r3 = (T)0.86602540378443864676;   // cos(pi/6)
        const T h = (T)0.5;                       // sin(pi/6)
        cx<T> b[4][3];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            b[n2][0] = a[n2];
            b[n2][1] = a[4 + n2];
            b[n2][2] = a[8 + n2];
            Dft<T, 3, DIR>::run(b[n2]);
        }
        // twiddles w12^{n2 k1}: exponents 1, 2 (n2 = 1), 2, 4 (n2 = 2), 3, 6 (n2 = 3)
        b[1][1] = mul_cs<T, DIR>(b[1][1], r3, h);
        b[1][2] = mul_cs<T, DIR>(b[1][2], h, r3);
        b[2][1] = mul_cs<T, DIR>(b[2][1], h, r3);
        b[2][2] = mul_cs<T, DIR>(b[2][2], -h, r3);
        b[3][1] = mul_i<T, DIR>(b[3][1]);
        b[3][2] = mkc<T>(-b[3][2].x, -b[3][2].y);
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            cx<T> c[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
            Dft<T, 4, DIR>::run(c);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[k1 + 3 * k2] = c[k2];
        }
    }
};

// ------------------------------------------------------------ line transform
__host__ __device__ constexpr int ce_min(int a, int b) { return a < b ? a : b; }
// Radix of the next stage for `rem` points left and E points per thread:
// 12 or 3 while a factor 3 remains, then the largest power of two that
// divides E (capped by rem).
__host__ __device__ constexpr int pick_radix(int rem, int E) {
    return (rem % 12 == 0 && E % 12 == 0) ? 12
           : (rem % 3 == 0 && E % 3 == 0) ? 3
                                          : ce_min(rem, E & -E);
}

template <int N> struct LinePad {
    // padded scratch index: one spare slot per 8 points
    __device__ __forceinline__ static int at(int pos) { return pos + (pos >> 3); }
    static constexpr int LEN = N + N / 8;
    // pitch between the lines of a warp: >= LEN and = 4 (mod 16)
    static constexpr int PITCH = LEN + ((4 - (LEN % 16)) + 16) % 16;
};

// Scratch policies.  WarpScratch: the line's threads are lanes of one warp
// and its scratch is contiguous (padded); exchanges need only __syncwarp.
// ColScratch: a block transforms many lines ("columns") at once, column z's
// point pos lives at (pad(pos)) * ld + z, so a warp of consecutive columns
// touches consecutive words; exchanges need __syncthreads.
template <typename T, int N> struct WarpScratch {
    cx<T> *base;
    __device__ __forceinline__ cx<T> &at(int pos) const { return base[LinePad<N>::at(pos)]; }
    __device__ __forceinline__ static void sync() { __syncwarp(); }
};
template <typename T, int N> struct ColScratch {
    cx<T> *base;   // already offset by the column index
    int ld;        // columns of the scratch
    __device__ __forceinline__ cx<T> &at(int pos) const { return base[(size_t)LinePad<N>::at(pos) * ld]; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};

template <typename T, int N, int E, int DIR, int NS, class S> struct LineStages {
    static constexpr int TPL = N / E;
    static constexpr int R = pick_radix(N / NS, E);
    static constexpr int B = E / R;              // butterflies per thread
    static constexpr bool LAST = (NS * R == N);
    static_assert(E % R == 0 && (N / NS) % R == 0, "radix must divide the points per thread and the rest");

    __device__ __forceinline__ static void run(cx<T> (&v)[E], int t, const S &scr, const cx<T> *tw) {
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int j = t + u * TPL;
            const int jm = j % NS;
            cx<T> bf[R];
#pragma unroll
            for (int r = 0; r < R; ++r) bf[r] = v[u + r * B];
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    cx<T> w = tw[jm * r * (N / (NS * R))];
                    if (DIR < 0) w.y = -w.y;
                    bf[r] = cmul<T>(bf[r], w);
                }
            }
            Dft<T, R, DIR>::run(bf);
            if (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[u + r * B] = bf[r];
            } else {
                const int base = (j / NS) * NS * R + jm;
#pragma unroll
                for (int r = 0; r < R; ++r) scr.at(base + r * NS) = bf[r];
            }
        }
        if (!LAST) {
            S::sync();
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = scr.at(t + e * TPL);
            S::sync();
            LineStages<T, N, E, DIR, NS * R, S>::run(v, t, scr, tw);
        }
    }
};

template <typename T, int N, int E, int DIR, class S> struct LineStages<T, N, E, DIR, N, S> {
    __device__ __forceinline__ static void run(cx<T> (&)[E], int, const S &, const cx<T> *) {}
};

// Transform one line held as described above.  `scr` is this line's scratch
// (LinePad<N>::LEN slots), `tw` the table exp(+2 pi i k / N), k < N.
template <typename T, int N, int E, int DIR>
__device__ __forceinline__ void line_fft(cx<T> (&v)[E], int t, cx<T> *scr, const cx<T> *tw) {
    WarpScratch<T, N> s{scr};
    LineStages<T, N, E, DIR, 1, WarpScratch<T, N>>::run(v, t, s, tw);
}

// Transform the column `z` of a block-wide set of columns: thread t of the
// column holds points t + e * (N / E); `scr` has LinePad<N>::LEN rows of
// `ld` columns.  Every thread of the block must call this together.
template <typename T, int N, int E, int DIR>
__device__ __forceinline__ void col_fft(cx<T> (&v)[E], int t, cx<T> *scr, int z, int ld, const cx<T> *tw) {
    ColScratch<T, N> s{scr + z, ld};
    LineStages<T, N, E, DIR, 1, ColScratch<T, N>>::run(v, t, s, tw);
}

// Points per thread by precision and length: 8, or 12 for lengths 3 * 2^a.
template <typename T, int N> struct LineCfg {
    static constexpr int E = N % 3 == 0 ? 12 : 8;
    static constexpr int TPL = N / E;
    static constexpr int LPW = 32 / TPL;
    static_assert(TPL >= 1 && TPL <= 32, "line must fit one warp");
};

// Points per thread of the forward transform's line kernels: 2 at N = 32 and
// 64 (radix-2 stages), 6 at N = 48 (a radix-3 stage, then radix 2): more
// threads per line than LineCfg (four times the warps at N = 64), since these
// passes have only N^2 / 2 to N^2 lines for the whole GPU; LineCfg's otherwise.
template <typename T, int N> struct FwdCfg {
    static constexpr int E = (N == 32 || N == 64) ? 2 : N == 48 ? 6 : LineCfg<T, N>::E;
    static constexpr int TPL = N / E;
    static constexpr int LPW = 32 / TPL;
    static_assert(TPL >= 1 && TPL <= 32, "line must fit one warp");
};

// 64-point inverse line transform of 4 lines per warp (lane = c + 4 t, thread
// t of line c holds x[t + 8 e] in v[e] and returns X[t + 8 e]): a radix-8
// DFT over e in registers, the twiddles w64^{t k1} (wt, per thread), an
// exchange through `slot` (256 complex entries, the warp's own) and a radix-8
// DFT over t.  Entry (t, k1) of the exchange sits at k1 * 32 + c + 4 (t ^ k1):
// the writes of one k1 and the transposed reads of one t both cover 16
// distinct 8-byte slots per half-warp, so neither has bank conflicts.
// `tws` is the table exp(2 pi i k / 64), k < 64 (shared memory).
__device__ __forceinline__ void line64_swz(float2 (&v)[8], int c, int t, float2 *__restrict__ slot,
                                           const float2 *__restrict__ tws) {
    Dft<float, 8, +1>::run(v);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = cmul<float>(v[k], tws[(t * k) & 63]);
#pragma unroll
    for (int k = 0; k < 8; ++k) slot[k * 32 + c + 4 * (t ^ k)] = v[k];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = slot[t * 32 + c + 4 * (r ^ t)];
    __syncwarp();
    Dft<float, 8, +1>::run(v);
}

}  // namespace wke
