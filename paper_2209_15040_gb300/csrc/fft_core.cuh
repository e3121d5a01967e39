// Register-resident pencil FFT core for sm_103a.
//
// One pencil of length N is spread over T = N/E threads, each holding E
// complex values in registers.  The transform is the self-sorting (Stockham)
// form of Cooley-Tukey: stage s combines R_s-point DFTs, multiplies by the
// roots of unity of that level, and writes its results in an order that
// leaves the final output in natural order.  This is the role the paper's
// even/odd "reshape" plays after each radix-2 level (Section 4.1), done here
// with radix-8/16 butterflies in registers and one shared-memory exchange
// between stages instead of a reshape per level.
//
// Stage s (radix R, Ns = product of the earlier radices), butterfly b in
// [0, N/R):   a[r] = X[b + r*N/R] * w_{Ns*R}^{r*(b mod Ns)},  a = DFT_R(a),
//             Y[(b div Ns)*Ns*R + (b mod Ns) + r*Ns] = a[r]
// with w_m = exp(-2*pi*i/m) (forward sign, Section 1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wsfft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// A float4 carries the same element of two adjacent pencils,
// (re0, im0, re1, im1); both halves get identical arithmetic and twiddles.
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 csub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 cmul(float4 a, float2 b) {
    return make_float4(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x), fmaf(a.z, b.x, -a.w * b.y),
                       fmaf(a.z, b.y, a.w * b.x));
}

// a * exp(-2*pi*i*J/16) for a compile-time J.  The constants are cos and sin
// of multiples of pi/8.
template <int J>
__device__ __forceinline__ float2 rot16(float2 a) {
    constexpr int j = ((J % 16) + 16) % 16;
    constexpr float H = 0.70710678118654752440f;   // cos(pi/4)
    constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return make_float2(a.y, -a.x);
    } else if constexpr (j == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (j == 12) {
        return make_float2(-a.y, a.x);
    } else if constexpr (j == 2) {
        return make_float2((a.x + a.y) * H, (a.y - a.x) * H);
    } else if constexpr (j == 6) {
        return make_float2((a.y - a.x) * H, -(a.x + a.y) * H);
    } else if constexpr (j == 10) {
        return make_float2(-(a.x + a.y) * H, (a.x - a.y) * H);
    } else if constexpr (j == 14) {
        return make_float2((a.x - a.y) * H, (a.x + a.y) * H);
    } else {
        // odd j: cos and sin of 2*pi*j/16 are +-cos(pi/8) or +-sin(pi/8)
        constexpr float c = (j == 1) ? C1 : (j == 3) ? S1 : (j == 5) ? -S1 : (j == 7) ? -C1
                          : (j == 9) ? -C1 : (j == 11) ? -S1 : (j == 13) ? S1 : C1;
        constexpr float s = (j == 1) ? S1 : (j == 3) ? C1 : (j == 5) ? C1 : (j == 7) ? S1
                          : (j == 9) ? -S1 : (j == 11) ? -C1 : (j == 13) ? -C1 : -S1;
        // (x + iy)(c - is) = (xc + ys) + i(yc - xs)
        return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
    }
}

// cos(j*pi/16), j in [0, 32), from the first-octant values by symmetry
__host__ __device__ constexpr double cos_pi16(int j) {
    j = ((j % 32) + 32) % 32;
    if (j > 16) j = 32 - j;              // cos(2pi - t) = cos t
    if (j > 8) return -cos_pi16(16 - j);  // cos(pi - t) = -cos t
    constexpr double base[9] = {1.0,
                                0.98078528040323044912618223613424,   // cos(pi/16)
                                0.92387953251128675612818318939679,   // cos(pi/8)
                                0.83146961230254523707878837761791,   // cos(3pi/16)
                                0.70710678118654752440084436210485,   // cos(pi/4)
                                0.55557023301960222474283081394853,   // cos(5pi/16)
                                0.38268343236508977172845998403040,   // cos(3pi/8)
                                0.19509032201612826784828486847702,   // cos(7pi/16)
                                0.0};
    return base[j];
}

// a * exp(-2*pi*i*J/32) for a compile-time J: even J reuses rot16
template <int J>
__device__ __forceinline__ float2 rot32(float2 a) {
    constexpr int j = ((J % 32) + 32) % 32;
    if constexpr (j % 2 == 0) {
        return rot16<j / 2>(a);
    } else {
        constexpr float c = (float)cos_pi16(j);
        constexpr float s = (float)cos_pi16(8 - j);  // sin(j*pi/16)
        return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
    }
}
template <int J>
__device__ __forceinline__ float4 rot32(float4 a) {
    const float2 lo = rot32<J>(make_float2(a.x, a.y)), hi = rot32<J>(make_float2(a.z, a.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int J>
__device__ __forceinline__ float4 rot16(float4 a) {
    const float2 lo = rot16<J>(make_float2(a.x, a.y)), hi = rot16<J>(make_float2(a.z, a.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// The same element of two adjacent pencils in split form: pencil 0 is
// (re.x, im.x), pencil 1 is (re.y, im.y).  Each real operation of the
// one-pencil butterfly becomes one packed FP32x2 instruction on the pair
// (sm_100 and later), with the same rounding in each lane, so the pair costs
// the instruction issue of a single pencil.
struct cpair {
    float2 re, im;
};
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ cpair cadd(cpair a, cpair b) {
    return {__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)};
}
__device__ __forceinline__ cpair csub(cpair a, cpair b) {
    return {__fadd2_rn(a.re, f2neg(b.re)), __fadd2_rn(a.im, f2neg(b.im))};
}
// one twiddle for both pencils; per lane exactly the float2 cmul above
__device__ __forceinline__ cpair cmul(cpair a, float2 w) {
    const float2 wr = f2dup(w.x), wi = f2dup(w.y);
    return {__ffma2_rn(a.re, wr, f2neg(__fmul2_rn(a.im, wi))), __ffma2_rn(a.re, wi, __fmul2_rn(a.im, wr))};
}

// rot16 on a split pair: per lane the same operations as the float2 version
template <int J>
__device__ __forceinline__ cpair rot16(cpair a) {
    constexpr int j = ((J % 16) + 16) % 16;
    constexpr float H = 0.70710678118654752440f;   // cos(pi/4)
    constexpr float C1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508977173f;  // sin(pi/8)
    const float2 h = f2dup(H);
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return {a.im, f2neg(a.re)};
    } else if constexpr (j == 8) {
        return {f2neg(a.re), f2neg(a.im)};
    } else if constexpr (j == 12) {
        return {f2neg(a.im), a.re};
    } else if constexpr (j == 2) {
        return {__fmul2_rn(__fadd2_rn(a.re, a.im), h), __fmul2_rn(__fadd2_rn(a.im, f2neg(a.re)), h)};
    } else if constexpr (j == 6) {
        return {__fmul2_rn(__fadd2_rn(a.im, f2neg(a.re)), h), f2neg(__fmul2_rn(__fadd2_rn(a.re, a.im), h))};
    } else if constexpr (j == 10) {
        return {f2neg(__fmul2_rn(__fadd2_rn(a.re, a.im), h)), __fmul2_rn(__fadd2_rn(a.re, f2neg(a.im)), h)};
    } else if constexpr (j == 14) {
        return {__fmul2_rn(__fadd2_rn(a.re, f2neg(a.im)), h), __fmul2_rn(__fadd2_rn(a.re, a.im), h)};
    } else {
        constexpr float c = (j == 1) ? C1 : (j == 3) ? S1 : (j == 5) ? -S1 : (j == 7) ? -C1
                          : (j == 9) ? -C1 : (j == 11) ? -S1 : (j == 13) ? S1 : C1;
        constexpr float s = (j == 1) ? S1 : (j == 3) ? C1 : (j == 5) ? C1 : (j == 7) ? S1
                          : (j == 9) ? -S1 : (j == 11) ? -C1 : (j == 13) ? -C1 : -S1;
        const float2 cc = f2dup(c), ss = f2dup(s);
        return {__ffma2_rn(a.re, cc, __fmul2_rn(a.im, ss)), __ffma2_rn(a.im, cc, f2neg(__fmul2_rn(a.re, ss)))};
    }
}
template <int J>
__device__ __forceinline__ cpair rot32(cpair a) {
    constexpr int j = ((J % 32) + 32) % 32;
    if constexpr (j % 2 == 0) {
        return rot16<j / 2>(a);
    } else {
        const float2 cc = f2dup((float)cos_pi16(j)), ss = f2dup((float)cos_pi16(8 - j));
        return {__ffma2_rn(a.re, cc, __fmul2_rn(a.im, ss)), __ffma2_rn(a.im, cc, f2neg(__fmul2_rn(a.re, ss)))};
    }
}

// In-register R-point forward DFT (R in {1,2,4,8,16,32}), natural order in and
// out: split into even and odd halves, transform each, combine with
// exp(-2*pi*i*k/R).
template <int R, int K, class V>
__device__ __forceinline__ void dft_combine(V (&a)[R], const V (&e)[R / 2], const V (&o)[R / 2]) {
    if constexpr (K < R / 2) {
        const V t = rot32<K * (32 / R)>(o[K]);
        a[K] = cadd(e[K], t);
        a[K + R / 2] = csub(e[K], t);
        dft_combine<R, K + 1>(a, e, o);
    }
}

template <int R, class V>
__device__ __forceinline__ void dft(V (&a)[R]) {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32, "radix");
    if constexpr (R == 2) {
        const V t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    } else if constexpr (R > 2) {
        V e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = a[2 * i];
            o[i] = a[2 * i + 1];
        }
        dft<R / 2>(e);
        dft<R / 2>(o);
        dft_combine<R, 0>(a, e, o);
    }
}

// Stage schedule for a pencil of length N with E values per thread: every
// stage has radix E except the last, whose radix is whatever remains.  The
// host plan builder calls the same functions to lay out the twiddle tables.
__host__ __device__ constexpr int sched_nstages(int N, int E) {
    int s = 0;
    long ns = 1;
    while (ns < N) {
        ns *= E;
        ++s;
    }
    return s < 1 ? 1 : s;
}
__host__ __device__ constexpr int sched_ns_before(int N, int E, int s) {
    long ns = 1;
    for (int i = 0; i < s; ++i) ns *= E;
    return ns > N ? N : (int)ns;
}
__host__ __device__ constexpr int sched_radix(int N, int E, int s) {
    return (N / sched_ns_before(N, E, s) < E) ? N / sched_ns_before(N, E, s) : E;
}
// stage s >= 1 reads twiddles tw[off(s) + (r-1)*Ns + k] = w_{Ns*R}^{r*k},
// r in [1,R), k in [0,Ns)
__host__ __device__ constexpr int sched_tw_offset(int N, int E, int s) {
    int off = 0;
    for (int i = 1; i < s; ++i) off += (sched_radix(N, E, i) - 1) * sched_ns_before(N, E, i);
    return off;
}
__host__ __device__ constexpr int sched_tw_size(int N, int E) {
    return sched_tw_offset(N, E, sched_nstages(N, E));
}

template <int N, int E>
struct Sched {
    static_assert(E >= 1 && E <= 32 && (E & (E - 1)) == 0, "E");
    static_assert(N >= E && (N & (N - 1)) == 0, "N");
    static constexpr int T = N / E;  // threads per pencil
    __host__ __device__ static constexpr int nstages() { return sched_nstages(N, E); }
    __host__ __device__ static constexpr int ns_before(int s) { return sched_ns_before(N, E, s); }
    __host__ __device__ static constexpr int radix(int s) { return sched_radix(N, E, s); }
    __host__ __device__ static constexpr int tw_offset(int s) { return sched_tw_offset(N, E, s); }
    __host__ __device__ static constexpr int tw_size() { return sched_tw_size(N, E); }
};

// Runs stages S_IDX.. of the pencil transform.  `a` holds the outputs of
// stage S_IDX-1 for this thread's butterflies.  Acc provides
//   gload(k), gstore(k, v)  -- global element k of this thread's pencil
//   sstore(k, v), sload(k)  -- shared-memory element k of the pencil
//   sync()                  -- barrier over every thread that shares the tile
//   after_load()            -- called once the first stage's inputs are in registers
// value type of an accessor: float2 (one pencil) unless it declares
// `using value_type = float4` (a pencil pair)
template <class Acc, class = void>
struct AccValue {
    using type = float2;
};
template <class Acc>
struct AccValue<Acc, decltype((void)sizeof(typename Acc::value_type), void())> {
    using type = typename Acc::value_type;
};

template <int N, int E, int S_IDX, class Acc, class V>
__device__ __forceinline__ void run_stages(V (&a)[E], Acc &acc, int t, const float2 *__restrict__ tw) {
    using S = Sched<N, E>;
    constexpr int T = S::T;
    constexpr int NsPrev = S::ns_before(S_IDX - 1);
    constexpr int Rprev = S::radix(S_IDX - 1);
    constexpr int Mprev = E / Rprev;
    if constexpr (S_IDX == S::nstages()) {
        // previous stage was the last: Ns*R == N, so its output index is b + r*Ns
#pragma unroll
        for (int i = 0; i < Mprev; ++i)
#pragma unroll
            for (int r = 0; r < Rprev; ++r) acc.gstore(t + T * i + r * NsPrev, a[i * Rprev + r]);
    } else {
#pragma unroll
        for (int i = 0; i < Mprev; ++i) {
            const int b = t + T * i;
            const int base = (b / NsPrev) * NsPrev * Rprev + (b % NsPrev);
#pragma unroll
            for (int r = 0; r < Rprev; ++r) acc.sstore(base + r * NsPrev, a[i * Rprev + r]);
        }
        acc.sync();
        constexpr int Ns = NsPrev * Rprev;
        constexpr int R = S::radix(S_IDX);
        constexpr int M = E / R;
        constexpr int TWO = S::tw_offset(S_IDX);
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int r = 0; r < R; ++r) a[i * R + r] = acc.sload(t + T * i + r * (N / R));
        acc.sync();
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int k = (t + T * i) % Ns;
            V g[R];
            g[0] = a[i * R];
#pragma unroll
            for (int r = 1; r < R; ++r) g[r] = cmul(a[i * R + r], __ldg(&tw[TWO + (r - 1) * Ns + k]));
            dft<R>(g);
#pragma unroll
            for (int r = 0; r < R; ++r) a[i * R + r] = g[r];
        }
        run_stages<N, E, S_IDX + 1>(a, acc, t, tw);
    }
}

// Whole pencil: first stage straight from global memory, last stage straight
// to global memory, shared-memory exchanges in between.
template <int N, int E, class Acc>
__device__ __forceinline__ void pencil_fft(Acc &acc, int t, const float2 *__restrict__ tw) {
    constexpr int T = Sched<N, E>::T;
    typename AccValue<Acc>::type a[E];
#pragma unroll
    for (int r = 0; r < E; ++r) a[r] = acc.gload(t + r * T);
    acc.after_load();
    dft<E>(a);
    run_stages<N, E, 1>(a, acc, t, tw);
}

// ---------------------------------------------------------------------------
// Storage conversion.  Reduced-precision values are widened to float32 on
// load and rounded to nearest-even on store.

// Cache operators for global accesses: default, .cg (L2 only: data another
// block may have written during this launch), .cs (streaming: read or
// written once, evict first).
enum : int { OP_DEF = 0, OP_CG = 1, OP_CS = 2 };

template <int OP, class T>
__device__ __forceinline__ T ld_op(const T *p) {
    if constexpr (OP == OP_CG) return __ldcg(p);
    else if constexpr (OP == OP_CS) return __ldcs(p);
    else return *p;
}
template <int OP, class T>
__device__ __forceinline__ void st_op(T *p, T v) {
    if constexpr (OP == OP_CS) __stcs(p, v);
    else *p = v;
}

template <class S>
struct Cvt;

template <>
struct Cvt<float2> {
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float2 load(const float2 *p) { return ld_op<OP>(p); }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(float2 *p, float2 v) { st_op<OP>(p, v); }
};

template <>
struct Cvt<__half2> {
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float2 load(const __half2 *p) {
        return __half22float2(ld_op<OP>(p));
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(__half2 *p, float2 v) {
        st_op<OP>(p, __float22half2_rn(v));
    }
};

template <>
struct Cvt<__nv_bfloat162> {
    template <int OP = OP_DEF>
    __device__ __forceinline__ static float2 load(const __nv_bfloat162 *p) {
        return __bfloat1622float2(ld_op<OP>(p));
    }
    template <int OP = OP_DEF>
    __device__ __forceinline__ static void store(__nv_bfloat162 *p, float2 v) {
        st_op<OP>(p, __float22bfloat162_rn(v));
    }
};

}  // namespace wsfft
