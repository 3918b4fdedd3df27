// Paired FP32 (y, z) plane convolution: the mixed form's hot FFT stage.
//
// Same mathematics as k_fft_yzc (zero-padded four-step FFT along z and y of
// one x-frequency plane, product with the real kernel spectrum, inverse,
// crop), restructured for Blackwell's paired FP32 instructions (add, sub,
// mul, fma on float2 = two lanes of one 64-bit register pair; one issue slot
// for two FP32 operations).  Every thread runs two independent sub-transforms
// side by side: a value CP holds the same element of transforms a and b,
// re = (re_a, re_b), im = (im_a, im_b), so every complex operation is a
// handful of paired instructions and no register is ever shuffled between
// halves.  The two transforms are
//   z passes: rows y = 2m and 2m + 1 (same sub-transform index, same twiddle);
//   y passes: columns kz = 2c and 2c + 1 (same twiddle; kernel values of the
//             two columns from the spectrum slice staged in shared memory).
// Shared memory is planar (separate re and im planes) so that the two values
// of a pair are adjacent and move with one 64-bit access:
//   Lz  (z phase): element (y, s) at (y / 2) * PZZ + 2 s + (y % 2);
//   Lq  (between the phases): as Lz with kz in even-odd order
//        s = kz / 2 + (kz % 2) * Mz / 2;
//   Ly  (y phase): element (y, kz) at y * Mz + kz.
// Within a phase every access is a 64-bit pair; where the phase changes (z to
// y and back) one side uses 32-bit accesses.  PZZ = 2 Mz + 2 keeps the z-phase
// accesses, whose lanes run over row pairs, on distinct banks; the lane maps
// below keep the others conflict-free too.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace sie {
namespace plane {

constexpr int kThreads = 256;

struct CP {
    float2 re, im;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n sub.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

__device__ __forceinline__ CP padd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP psub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// a * (C + i S) and a * (C - i S) for twiddle pairs (C, S)
__device__ __forceinline__ CP pmul(CP a, float2 C, float2 S) {
    return CP{sub2(mul2(a.re, C), mul2(a.im, S)), fma2(a.re, S, mul2(a.im, C))};
}
__device__ __forceinline__ CP pmulc(CP a, float2 C, float2 S) {
    return CP{fma2(a.im, S, mul2(a.re, C)), sub2(mul2(a.im, C), mul2(a.re, S))};
}

// cos and sin of 2 pi t / 16 for t = 0..15
__host__ __device__ constexpr double c16t(int t) {
    constexpr double c[16] = {1.0,
                              0.92387953251128675613,
                              0.70710678118654752440,
                              0.38268343236508977173,
                              0.0,
                              -0.38268343236508977173,
                              -0.70710678118654752440,
                              -0.92387953251128675613,
                              -1.0,
                              -0.92387953251128675613,
                              -0.70710678118654752440,
                              -0.38268343236508977173,
                              0.0,
                              0.38268343236508977173,
                              0.70710678118654752440,
                              0.92387953251128675613};
    return c[t & 15];
}
__host__ __device__ constexpr double s16t(int t) { return c16t(t - 4); }

// v * W_16^t, W = exp(-2 pi i / 16) (forward) or its conjugate (inverse);
// t is a compile-time constant after unrolling.
template <bool INV>
__device__ __forceinline__ CP ptw16(CP v, int t) {
    t &= 15;
    if (t == 0) return v;
    if (t == 4 || t == 12) {   // -i or +i (forward), swapped for the inverse
        const bool mi = (t == 4) != INV;
        const float2 z = dup2(0.f);
        return mi ? CP{v.im, sub2(z, v.re)} : CP{sub2(z, v.im), v.re};
    }
    if (t == 8) return CP{sub2(dup2(0.f), v.re), sub2(dup2(0.f), v.im)};
    const float c = float(c16t(t)), s = INV ? float(s16t(t)) : -float(s16t(t));
    return pmul(v, dup2(c), dup2(s));
}

// radix-4 butterfly in place: (a0, a1, a2, a3) -> DFT_4
template <bool INV>
__device__ __forceinline__ void pbfly4(CP &a0, CP &a1, CP &a2, CP &a3) {
    const CP t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
    a0 = padd(t0, t2);
    a2 = psub(t0, t2);
    if (!INV) {   // t1 -/+ i d
        a1 = CP{add2(t1.re, d.im), sub2(t1.im, d.re)};
        a3 = CP{sub2(t1.re, d.im), add2(t1.im, d.re)};
    } else {
        a1 = CP{sub2(t1.re, d.im), add2(t1.im, d.re)};
        a3 = CP{add2(t1.re, d.im), sub2(t1.im, d.re)};
    }
}

// In-register DFT of length N (2, 4, 8, 16) on v[0..N), natural order in and out.
// Inputs known to be zero (compile-time) fold away.
template <int N, bool INV>
__device__ __forceinline__ void pdft(CP (&v)[16]) {
    if constexpr (N == 2) {
        const CP a = v[0], b = v[1];
        v[0] = padd(a, b);
        v[1] = psub(a, b);
    } else if constexpr (N == 4) {
        pbfly4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (N == 8) {
        // n = j + 2 m: DFT_4 over m for j = 0, 1; twiddle W_8^(j k1); DFT_2 over j
        pbfly4<INV>(v[0], v[2], v[4], v[6]);
        pbfly4<INV>(v[1], v[3], v[5], v[7]);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[1 + 2 * k1] = ptw16<INV>(v[1 + 2 * k1], 2 * k1);
        CP o[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            o[k1] = padd(v[2 * k1], v[2 * k1 + 1]);
            o[k1 + 4] = psub(v[2 * k1], v[2 * k1 + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = o[i];
    } else {
        static_assert(N == 16, "DFT length");
        // n = j + 4 m: DFT_4 over m for each j; twiddle W_16^(j k1); DFT_4 over j
#pragma unroll
        for (int j = 0; j < 4; ++j) pbfly4<INV>(v[j], v[j + 4], v[j + 8], v[j + 12]);
#pragma unroll
        for (int j = 1; j < 4; ++j)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) v[j + 4 * k1] = ptw16<INV>(v[j + 4 * k1], j * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) pbfly4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
        CP o[16];   // v[4 k1 + k2] = X[k1 + 4 k2]
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
}

// DFT of length N whose inputs v[N/2 .. N) are zero (the zero-padded first
// stage of a forward transform), natural order in and out: the even outputs
// are the half-length DFT of v[0 .. N/2), the odd ones that of v[j] W_N^j.
template <int N>
__device__ __forceinline__ void pdft_zpad(CP (&v)[16]) {
    constexpr int H = N / 2;
    if constexpr (N == 2) {
        v[1] = v[0];
    } else {
        CP e[16], o[16];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            e[j] = v[j];
            o[j] = j ? ptw16<false>(v[j], j * (16 / N)) : v[j];
        }
        pdft<H, false>(e);
        pdft<H, false>(o);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            v[2 * m] = e[m];
            v[2 * m + 1] = o[m];
        }
    }
}

// The first N/2 outputs of the inverse DFT of length N (the cropped last
// stage of an inverse transform): out[p] = E[p] + W_N^-p O[p] with E and O the
// half-length inverse DFTs of the even and odd inputs.
template <int N>
__device__ __forceinline__ void pidft_half(CP (&v)[16]) {
    constexpr int H = N / 2;
    if constexpr (N == 2) {
        v[0] = padd(v[0], v[1]);
    } else {
        CP e[16], o[16];
#pragma unroll
        for (int m = 0; m < H; ++m) {
            e[m] = v[2 * m];
            o[m] = v[2 * m + 1];
        }
        pdft<H, true>(e);
        pdft<H, true>(o);
#pragma unroll
        for (int p = 0; p < H; ++p) v[p] = padd(e[p], p ? ptw16<true>(o[p], p * (16 / N)) : o[p]);
    }
}

__host__ __device__ constexpr int split_n1(int M) {
    int lg = 0;
    while ((1 << lg) < M) ++lg;
    return 1 << (lg / 2);
}
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Compile-time geometry of a padded My x Mz plane.
template <int MY, int MZ> struct Geo {
    static constexpr int Ny = MY / 2, Nz = MZ / 2, NYP = Ny / 2;   // input extent, row pairs
    static constexpr int A1 = split_n1(MZ), A2 = MZ / A1;           // z: Mz = A1 A2
    static constexpr int B1 = split_n1(MY), B2 = MY / B1;           // y: My = B1 B2
    static constexpr int PZZ = 2 * MZ + 2;                          // Lz / Lq row-pair pitch
    static constexpr int NP = cmax(NYP * PZZ, MY * MZ);             // floats per plane of P
    static constexpr int NQ = NYP * PZZ;                            // floats per plane of Q
    static constexpr int HSP = MZ / 2 + 2;                          // staged spectrum row pitch
    static constexpr int NH = ((MY / 2 + 1) * HSP + 1) / 2 * 2;     // staged spectrum (floats, even)
    static constexpr int NTW = 2 * (MY + MZ);                       // staged twiddles (float2)
    static constexpr size_t kSmem = size_t(2 * NP + 2 * NQ + NH) * sizeof(float) + size_t(NTW) * sizeof(float2);
    static_assert(NYP >= 1 && A1 >= 2 && A2 >= 2 && B1 >= 2 && B2 >= 2 && A2 <= 16 && B2 <= 16, "plane size");
};


__device__ __forceinline__ float2 &at2(float *base, int i) { return *reinterpret_cast<float2 *>(base + i); }
__device__ __forceinline__ float2 ld2(const float *base, int i) { return *reinterpret_cast<const float2 *>(base + i); }

// Row-pair index of z-pass item u with G = 16 / A2 row pairs per half-warp:
// the G row pairs of a half-warp are spaced A2 apart so that, at row-pair pitch
// PZZ = 2 (mod 8), their 64-bit accesses cover distinct banks.
template <int NYP, int A2>
__device__ __forceinline__ int zrow(int u) {
    constexpr int G = 16 / A2;
    if constexpr (G >= 2 && NYP % 16 == 0) {
        const int q = u % G, r = (u / G) % A2, hi = u / 16;
        return hi * 16 + q * A2 + r;
    } else {
        return u;
    }
}

// Item (c, j) of a y pass over NC column pairs and J sub-transforms: with
// NC >= 16 a warp takes 16 column pairs of two consecutive j (rows of
// opposite parity), so the 32-bit accesses to Lq of its two half-warps fall on
// even and odd banks respectively.
template <int NC>
__device__ __forceinline__ void ycol(int it, int &c, int &j) {
    if constexpr (NC >= 16) {
        const int lo = it % 16, b = (it / 16) % 2, r = it / 32;
        c = lo + 16 * (r % (NC / 16));
        j = 2 * (r / (NC / 16)) + b;
    } else {
        c = it % NC;
        j = it / NC;
    }
}

// F1: z pass 1 of rows y < Ny (input z < Nz), global -> P (Lz), slot j2 + A2 k1;
// tw = W_Mz^(j2 k1) stored [k1][j2].  The global loads are split off (f1_load)
// so that a CTA issues the next plane's loads while it finishes the current one.
template <int MY, int MZ> struct F1In {
    static constexpr int kItems = (Geo<MY, MZ>::NYP * Geo<MY, MZ>::A2 + kThreads - 1) / kThreads;
    float2 a[kItems][Geo<MY, MZ>::A1 / 2], b[kItems][Geo<MY, MZ>::A1 / 2];   // rows 2m, 2m + 1
};
template <int MY, int MZ>
__device__ __forceinline__ void f1_load(const float2 *__restrict__ src, F1In<MY, MZ> &in) {
    using G = Geo<MY, MZ>;
    constexpr int A2 = G::A2, H1 = G::A1 / 2;
#pragma unroll
    for (int q = 0; q < F1In<MY, MZ>::kItems; ++q) {
        const int it = threadIdx.x + q * kThreads;
        if (it < G::NYP * A2) {
            const int j2 = it % A2, m = zrow<G::NYP, A2>(it / A2);
            const float2 *r0 = src + (2 * m) * G::Nz + j2, *r1 = r0 + G::Nz;
#pragma unroll
            for (int j1 = 0; j1 < H1; ++j1) {
                in.a[q][j1] = __ldg(r0 + A2 * j1);
                in.b[q][j1] = __ldg(r1 + A2 * j1);
            }
        }
    }
}
template <int MY, int MZ>
__device__ __forceinline__ void f1(const F1In<MY, MZ> &in, float *Pre, float *Pim, const float2 *tw) {
    using G = Geo<MY, MZ>;
    constexpr int A1 = G::A1, A2 = G::A2, H1 = A1 / 2;
#pragma unroll
    for (int q = 0; q < F1In<MY, MZ>::kItems; ++q) {
        const int it = threadIdx.x + q * kThreads;
        if (it >= G::NYP * A2) break;
        const int j2 = it % A2, m = zrow<G::NYP, A2>(it / A2);
        CP v[16];
#pragma unroll
        for (int j1 = 0; j1 < H1; ++j1) {
            const float2 a = in.a[q][j1], b = in.b[q][j1];
            v[j1] = CP{make_float2(a.x, b.x), make_float2(a.y, b.y)};
        }
        pdft_zpad<A1>(v);   // inputs j1 >= A1 / 2 are the zero padding
#pragma unroll
        for (int k1 = 0; k1 < A1; ++k1) {
            CP o = v[k1];
            if (k1) {
                const float2 w = tw[k1 * A2 + j2];
                o = pmul(o, dup2(w.x), dup2(w.y));
            }
            const int i = m * G::PZZ + 2 * (j2 + A2 * k1);
            at2(Pre, i) = o.re;
            at2(Pim, i) = o.im;
        }
    }
}

// F2: z pass 2, P (Lz) -> Q (Lq), natural kz = k1 + A1 k2.
template <int MY, int MZ>
__device__ __forceinline__ void f2(const float *Pre, const float *Pim, float *Qre, float *Qim) {
    using G = Geo<MY, MZ>;
    constexpr int A1 = G::A1, A2 = G::A2;
    for (int it = threadIdx.x; it < G::NYP * A1; it += kThreads) {
        const int m = it % G::NYP, k1 = it / G::NYP;
        CP v[16];
#pragma unroll
        for (int j2 = 0; j2 < A2; ++j2) {
            const int i = m * G::PZZ + 2 * (j2 + A2 * k1);
            v[j2] = CP{ld2(Pre, i), ld2(Pim, i)};
        }
        pdft<A2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < A2; ++k2) {
            const int kz = k1 + A1 * k2;
            const int i = m * G::PZZ + 2 * ((kz >> 1) + (kz & 1) * (MZ / 2));
            at2(Qre, i) = v[k2].re;
            at2(Qim, i) = v[k2].im;
        }
    }
}

// F3: y pass 1 of column pairs (2c, 2c + 1), Q (Lq, rows y < Ny) -> P (Ly), row k1 B2 + j2.
template <int MY, int MZ>
__device__ __forceinline__ void f3(const float *Qre, const float *Qim, float *Pre, float *Pim, const float2 *tw) {
    using G = Geo<MY, MZ>;
    constexpr int B1 = G::B1, B2 = G::B2, H1 = B1 / 2, NC = MZ / 2;
    for (int it = threadIdx.x; it < NC * B2; it += kThreads) {
        int c, j2;
        ycol<NC>(it, c, j2);
        CP v[16];
#pragma unroll
        for (int j1 = 0; j1 < H1; ++j1) {
            const int y = j2 + B2 * j1;
            const int i0 = (y >> 1) * G::PZZ + 2 * c + (y & 1), i1 = i0 + MZ;   // kz = 2c, 2c + 1
            v[j1] = CP{make_float2(Qre[i0], Qre[i1]), make_float2(Qim[i0], Qim[i1])};
        }
        pdft_zpad<B1>(v);   // rows y >= N_y are the zero padding
#pragma unroll
        for (int k1 = 0; k1 < B1; ++k1) {
            CP o = v[k1];
            if (k1) {
                const float2 w = tw[j2 * B1 + k1];
                o = pmul(o, dup2(w.x), dup2(w.y));
            }
            const int i = (k1 * B2 + j2) * MZ + 2 * c;
            at2(Pre, i) = o.re;
            at2(Pim, i) = o.im;
        }
    }
}

// y pass 2, times H(kx, ky, kz), inverse y pass A, in place on P (Ly): rows
// k1 B2 + j2 in, rows k1 + B1 p2 out.  A round takes CW = kThreads / B1 column
// pairs with all their k1, so every read of a column precedes every write.
// Hs: this kx's spectrum staged in shared memory, [fold(ky)][hz(fold(kz))] with
// row pitch HSP and hz(f) = f + (f == Mz/2): the two loads of a column pair
// then hit distinct banks (lanes c and Mz/2 - c share words).
template <int MZ>
__device__ __forceinline__ int hz_slot(int kz) {
    const int f = kz <= MZ / 2 ? kz : MZ - kz;
    return f + (f == MZ / 2 ? 1 : 0);
}
template <int MY, int MZ>
__device__ __forceinline__ void ymid(float *Pre, float *Pim, const float *Hs, const float2 *twi) {
    using G = Geo<MY, MZ>;
    constexpr int B1 = G::B1, B2 = G::B2, NC = MZ / 2, CW = kThreads / B1;
    const int k1 = threadIdx.x / CW, cl = threadIdx.x % CW;
    for (int c0 = 0; c0 < NC; c0 += CW) {
        const int c = c0 + cl;
        const bool act = k1 < B1 && c < NC;
        CP v[16];
        if (act) {
#pragma unroll
            for (int j2 = 0; j2 < B2; ++j2) {
                const int i = (k1 * B2 + j2) * MZ + 2 * c;
                v[j2] = CP{ld2(Pre, i), ld2(Pim, i)};
            }
            pdft<B2, false>(v);   // v[k2] = X[ky = k1 + B1 k2]
#pragma unroll
            for (int k2 = 0; k2 < B2; ++k2) {
                const int ky = k1 + B1 * k2, fy = ky <= MY / 2 ? ky : MY - ky;
                const float *hr = Hs + fy * G::HSP;
                const float2 h = make_float2(hr[hz_slot<MZ>(2 * c)], hr[hz_slot<MZ>(2 * c + 1)]);
                v[k2] = CP{mul2(v[k2].re, h), mul2(v[k2].im, h)};
            }
            pdft<B2, true>(v);
#pragma unroll
            for (int p2 = 1; p2 < B2; ++p2) {
                const float2 w = twi[k1 * B2 + p2];
                v[p2] = pmulc(v[p2], dup2(w.x), dup2(w.y));
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int p2 = 0; p2 < B2; ++p2) {
                const int i = (k1 + B1 * p2) * MZ + 2 * c;
                at2(Pre, i) = v[p2].re;
                at2(Pim, i) = v[p2].im;
            }
        }
        __syncthreads();
    }
}

// I2: inverse y pass B of column pairs, P (Ly, rows p2 B1 + k1) -> Q (Lq, rows
// y = p2 + B2 p1 < Ny).
template <int MY, int MZ>
__device__ __forceinline__ void i2(const float *Pre, const float *Pim, float *Qre, float *Qim) {
    using G = Geo<MY, MZ>;
    constexpr int B1 = G::B1, B2 = G::B2, H1 = B1 / 2, NC = MZ / 2;
    for (int it = threadIdx.x; it < NC * B2; it += kThreads) {
        int c, p2;
        ycol<NC>(it, c, p2);
        CP v[16];
#pragma unroll
        for (int k1 = 0; k1 < B1; ++k1) {
            const int i = (p2 * B1 + k1) * MZ + 2 * c;
            v[k1] = CP{ld2(Pre, i), ld2(Pim, i)};
        }
        pidft_half<B1>(v);   // only rows y < N_y are kept
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) {
            const int y = p2 + B2 * p1;
            const int i0 = (y >> 1) * G::PZZ + 2 * c + (y & 1), i1 = i0 + MZ;   // kz = 2c, 2c + 1
            Qre[i0] = v[p1].re.x;
            Qre[i1] = v[p1].re.y;
            Qim[i0] = v[p1].im.x;
            Qim[i1] = v[p1].im.y;
        }
    }
}

// I3: inverse z pass A of rows y < Ny, Q (Lq, kz = k1 + A1 k2) -> P (Lz), slot p2 + A2 k1.
template <int MY, int MZ>
__device__ __forceinline__ void i3(const float *Qre, const float *Qim, float *Pre, float *Pim, const float2 *twi) {
    using G = Geo<MY, MZ>;
    constexpr int A1 = G::A1, A2 = G::A2;
    for (int it = threadIdx.x; it < G::NYP * A1; it += kThreads) {
        const int m = it % G::NYP, k1 = it / G::NYP;
        CP v[16];
#pragma unroll
        for (int k2 = 0; k2 < A2; ++k2) {
            const int kz = k1 + A1 * k2;
            const int i = m * G::PZZ + 2 * ((kz >> 1) + (kz & 1) * (MZ / 2));
            v[k2] = CP{ld2(Qre, i), ld2(Qim, i)};
        }
        pdft<A2, true>(v);
#pragma unroll
        for (int p2 = 0; p2 < A2; ++p2) {
            CP o = v[p2];
            if (p2) {
                const float2 w = twi[k1 * A2 + p2];
                o = pmulc(o, dup2(w.x), dup2(w.y));
            }
            const int i = m * G::PZZ + 2 * (p2 + A2 * k1);
            at2(Pre, i) = o.re;
            at2(Pim, i) = o.im;
        }
    }
}

// I4: inverse z pass B, P (Lz) -> global rows y < Ny, z = p2 + A2 p1 < Nz.
template <int MY, int MZ>
__device__ __forceinline__ void i4(const float *Pre, const float *Pim, float2 *__restrict__ dst) {
    using G = Geo<MY, MZ>;
    constexpr int A1 = G::A1, A2 = G::A2, H1 = A1 / 2;
    for (int it = threadIdx.x; it < G::NYP * A2; it += kThreads) {
        const int p2 = it % A2, m = zrow<G::NYP, A2>(it / A2);
        CP v[16];
#pragma unroll
        for (int k1 = 0; k1 < A1; ++k1) {
            const int i = m * G::PZZ + 2 * (p2 + A2 * k1);
            v[k1] = CP{ld2(Pre, i), ld2(Pim, i)};
        }
        pidft_half<A1>(v);   // only z < N_z is kept
        float2 *r0 = dst + (2 * m) * G::Nz + p2, *r1 = r0 + G::Nz;
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) {
            r0[A2 * p1] = make_float2(v[p1].re.x, v[p1].im.x);
            r1[A2 * p1] = make_float2(v[p1].re.y, v[p1].im.y);
        }
    }
}

// The (y, z) part of the 3-D convolution, in place on planes [Ny][Nz] of the
// buffer [ngrids][Mx][Ny][Nz] (complex64).  One CTA per (kx, run of up to G
// grids): the kx slice of the spectrum and the four-step twiddles are staged
// in shared memory once and serve every plane of the run.
// Hp: spectrum [fold(kx)][fold(ky)][fold(kz)], scaled by 1/(Mx My Mz);
// tf[j2 N1 + k1] = W^(j2 k1), ti[k1 N2 + p2] = W^(k1 p2) (applied conjugated)
// for axis y (tfy, tiy) and z (tfz, tiz).
template <int MY, int MZ>
__global__ void __launch_bounds__(kThreads, 2)
    k_plane_conv(float2 *__restrict__ buf, int ngrids, int gpc, int lgMx, const float *__restrict__ Hp,
                 const float2 *__restrict__ tfy, const float2 *__restrict__ tiy, const float2 *__restrict__ tfz,
                 const float2 *__restrict__ tiz) {
    using G = Geo<MY, MZ>;
    extern __shared__ __align__(16) float psm[];
    float *Pre = psm, *Pim = psm + G::NP, *Qre = psm + 2 * G::NP, *Qim = Qre + G::NQ;
    float *Hs = Qim + G::NQ;
    float2 *s_tfy = reinterpret_cast<float2 *>(Hs + G::NH), *s_tiy = s_tfy + MY, *s_tfz = s_tiy + MY,
           *s_tiz = s_tfz + MZ;
    const int Mx = 1 << lgMx;
    const int kx = blockIdx.x & (Mx - 1), fx = kx <= Mx / 2 ? kx : Mx - kx;
    const int b0 = (blockIdx.x >> lgMx) * gpc, b1 = min(ngrids, b0 + gpc);
    {
        constexpr int HY = MY / 2 + 1, HZ = MZ / 2 + 1;
        const float *Hk = Hp + int64_t(fx) * HY * HZ;
        for (int i = threadIdx.x; i < HY * HZ; i += kThreads) {
            const int fy = i / HZ, fz = i - fy * HZ;
            Hs[fy * G::HSP + fz + (fz == MZ / 2 ? 1 : 0)] = __ldg(Hk + i);
        }
        for (int i = threadIdx.x; i < MY; i += kThreads) {
            s_tfy[i] = __ldg(tfy + i);
            s_tiy[i] = __ldg(tiy + i);
        }
        for (int i = threadIdx.x; i < MZ; i += kThreads) {
            // F1 reads W^(j2 k1) with lanes over j2: stored [k1][j2]
            const int j2 = i / G::A1, k1 = i - j2 * G::A1;
            s_tfz[k1 * G::A2 + j2] = __ldg(tfz + i);
            s_tiz[i] = __ldg(tiz + i);
        }
    }
    const int64_t pstride = int64_t(Mx) * G::Ny * G::Nz;
    F1In<MY, MZ> in;
    if (b0 < b1) f1_load<MY, MZ>(buf + int64_t(b0) * pstride + int64_t(kx) * G::Ny * G::Nz, in);
    __syncthreads();
    for (int b = b0; b < b1; ++b) {
        float2 *plane = buf + int64_t(b) * pstride + int64_t(kx) * G::Ny * G::Nz;
        f1<MY, MZ>(in, Pre, Pim, s_tfz);
        __syncthreads();
        f2<MY, MZ>(Pre, Pim, Qre, Qim);
        __syncthreads();
        f3<MY, MZ>(Qre, Qim, Pre, Pim, s_tfy);
        __syncthreads();
        ymid<MY, MZ>(Pre, Pim, Hs, s_tiy);
        i2<MY, MZ>(Pre, Pim, Qre, Qim);
        __syncthreads();
        if (b + 1 < b1) f1_load<MY, MZ>(plane + pstride, in);   // next plane, in flight during I3 and I4
        i3<MY, MZ>(Qre, Qim, Pre, Pim, s_tiz);
        __syncthreads();
        i4<MY, MZ>(Pre, Pim, plane);
        __syncthreads();
    }
}

}  // namespace plane
}  // namespace sie
