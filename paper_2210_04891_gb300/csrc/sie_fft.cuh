// Shared-memory Stockham FFT building blocks for the pFFT convolution
// (Sec. IV-B, step 2: the 3-level Toeplitz product H Q_g evaluated as an
// aperiodic convolution on the 2N_x x 2N_y x 2N_z zero-padded grid).
//
// A 1-D FFT of power-of-two length M over a batch of lines held in shared
// memory runs as log_R(M) Stockham stages (radix 4, one radix-2 stage when
// log2 M is odd).  In a stage each butterfly j in [0, M/R) reads
// x[j + r M/R], applies the twiddle W_M^(r (j mod Ns) M/(Ns R)), does an R-point
// DFT and writes y[(j div Ns) Ns R + (j mod Ns) + r Ns]; all threads first load
// their butterflies into registers, synchronise, then store in place, so a
// single buffer suffices.  Twiddles come from a table W[m] = exp(-2 pi i m / M).
#pragma once

#include "sie_common.cuh"

namespace sie {

constexpr int FFT_E = 16;   // elements per thread per stage (registers)

template <typename T>
__device__ __forceinline__ void dft4(C<T> &a0, C<T> &a1, C<T> &a2, C<T> &a3, bool inv) {
    C<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi(csub(a1, a3), inv);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// Batched in-place FFT of `nlines` lines of length M in shared memory `s`.
// Element e of line l sits at s[l * ls + e * es].  `lines_fast` maps
// consecutive threads to consecutive lines (use when ls == 1) instead of
// consecutive butterflies (use when es == 1), to keep shared accesses
// conflict-free.  Requires nlines * M <= FFT_E * blockDim.x.
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

template <typename T>
__device__ void fft_lines(C<T> *s, int M, int nlines, int ls, int es, const C<T> *__restrict__ tw, bool inv,
                          bool lines_fast) {
    // every size is a power of two: index arithmetic by shifts and masks
    const int lgM = ilog2(M), lgL = ilog2(nlines);
    int lgNs = 0;
    while (lgNs < lgM) {
        const int lgR = (lgM - lgNs >= 2) ? 2 : 1;
        const int R = 1 << lgR;
        const int Ns = 1 << lgNs;
        const int lgnbf = lgM - lgR;             // butterflies per line = M / R
        const int total = nlines << lgnbf;
        const int lgstep = lgM - lgNs - lgR;     // twiddle stride M / (Ns R)
        C<T> v[FFT_E];
#pragma unroll
        for (int i = 0; i < FFT_E / 2; ++i) {   // at most FFT_E/R butterflies, R >= 2
            const int it = threadIdx.x + i * blockDim.x;
            if (i * blockDim.x >= total) break;
            if (it < total && i * R < FFT_E) {
                int line, j;
                if (lines_fast) { line = it & (nlines - 1); j = it >> lgL; }
                else { j = it & ((1 << lgnbf) - 1); line = it >> lgnbf; }
                const C<T> *b = s + line * ls;
                const int jm = j & (Ns - 1);
                const int nbf = 1 << lgnbf;
                if (R == 4) {
                    C<T> a0 = b[j * es], a1 = b[(j + nbf) * es], a2 = b[(j + 2 * nbf) * es], a3 = b[(j + 3 * nbf) * es];
                    if (jm) {
                        const int t1 = jm << lgstep;
                        C<T> w1 = tw[t1], w2 = tw[2 * t1], w3 = tw[3 * t1];
                        if (inv) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
                        a1 = cmul(a1, w1); a2 = cmul(a2, w2); a3 = cmul(a3, w3);
                    }
                    dft4<T>(a0, a1, a2, a3, inv);
                    v[4 * i] = a0; v[4 * i + 1] = a1; v[4 * i + 2] = a2; v[4 * i + 3] = a3;
                } else {
                    C<T> a0 = b[j * es], a1 = b[(j + nbf) * es];
                    if (jm) {
                        C<T> w1 = tw[jm << lgstep];
                        if (inv) w1.y = -w1.y;
                        a1 = cmul(a1, w1);
                    }
                    v[2 * i] = cadd(a0, a1);
                    v[2 * i + 1] = csub(a0, a1);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < FFT_E / 2; ++i) {
            const int it = threadIdx.x + i * blockDim.x;
            if (i * blockDim.x >= total) break;
            if (it < total && i * R < FFT_E) {
                int line, j;
                if (lines_fast) { line = it & (nlines - 1); j = it >> lgL; }
                else { j = it & ((1 << lgnbf) - 1); line = it >> lgnbf; }
                C<T> *b = s + line * ls;
                const int d = ((j >> lgNs) << (lgNs + lgR)) + (j & (Ns - 1));
                if (R == 4) {
                    b[d * es] = v[4 * i]; b[(d + Ns) * es] = v[4 * i + 1];
                    b[(d + 2 * Ns) * es] = v[4 * i + 2]; b[(d + 3 * Ns) * es] = v[4 * i + 3];
                } else {
                    b[d * es] = v[2 * i]; b[(d + Ns) * es] = v[2 * i + 1];
                }
            }
        }
        __syncthreads();
        lgNs += lgR;
    }
}

// 2-D FFT of planes (y, z) held in shared memory, one plane per CTA.
// Input plane: [ny_in][nz_in] at src + blockIdx.x * src_stride (zero-padded to
// My x Mz); output plane: [ny_out][nz_out] at dst + blockIdx.x * dst_stride.
// Forward: z-FFT of rows y < ny_in, then y-FFT of all columns.
// Inverse: y-FFT of all columns, then z-FFT of rows y < ny_out.
template <typename T>
__global__ void __launch_bounds__(512) k_fft_plane(const C<T> *__restrict__ src, int64_t src_stride, int ny_in, int nz_in,
                            C<T> *__restrict__ dst, int64_t dst_stride, int ny_out, int nz_out, int My, int Mz,
                            const C<T> *__restrict__ tw_y, const C<T> *__restrict__ tw_z, int inverse) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *s = reinterpret_cast<C<T> *>(smem_raw);
    const C<T> *in = src + blockIdx.x * src_stride;
    const int P = My * Mz;
    const int lgMz = ilog2(Mz), lgnzi = ilog2(nz_in), lgnzo = ilog2(nz_out);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int y = i >> lgMz, z = i & (Mz - 1);
        s[i] = (y < ny_in && z < nz_in) ? in[(y << lgnzi) + z] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    if (!inverse) {
        fft_lines<T>(s, Mz, ny_in, Mz, 1, tw_z, false, false);
        fft_lines<T>(s, My, Mz, 1, Mz, tw_y, false, true);
    } else {
        fft_lines<T>(s, My, Mz, 1, Mz, tw_y, true, true);
        fft_lines<T>(s, Mz, ny_out, Mz, 1, tw_z, true, false);
    }
    C<T> *out = dst + blockIdx.x * dst_stride;
    for (int i = threadIdx.x; i < ny_out * nz_out; i += blockDim.x) {
        int y = i >> lgnzo, z = i & (nz_out - 1);
        out[i] = s[(y << lgMz) + z];
    }
}

__host__ __device__ __forceinline__ int fold_index(int k, int M) { return k <= M / 2 ? k : M - k; }

// FFT along x of pencils: buffer [batch][x][ncols] (x stride ncols), one CTA
// per (batch, tile of KT consecutive columns).  Loads x < nx_in (zero above),
// forward FFT; if H != nullptr multiplies by the real kernel spectrum
// H[fold(ky)][fold(kz)][fold(kx)] (column = ky * Mz + kz; fold(k) = min(k, M - k),
// the spectrum of an even kernel is even in each index) and runs the inverse
// FFT; stores x < nx_out in place.
template <typename T>
__global__ void __launch_bounds__(512) k_fft_pencil(C<T> *__restrict__ buf, int64_t batch_stride, int ncols, int nx_in, int nx_out,
                             int Mx, int My, int Mz, int KT, const C<T> *__restrict__ tw_x,
                             const T *__restrict__ H) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *s = reinterpret_cast<C<T> *>(smem_raw);
    const int tiles = ncols / KT;
    const int b = blockIdx.x / tiles, c0 = (blockIdx.x % tiles) * KT;
    C<T> *base = buf + b * batch_stride + c0;
    const int pitch = Mx + 1;
    const int lgKT = ilog2(KT), lgMx = ilog2(Mx), lgMz = ilog2(Mz);
    for (int i = threadIdx.x; i < KT * Mx; i += blockDim.x) {
        int x = i >> lgKT, c = i & (KT - 1);
        s[c * pitch + x] = x < nx_in ? base[int64_t(x) * ncols + c] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    fft_lines<T>(s, Mx, KT, pitch, 1, tw_x, false, false);
    if (H) {
        const int hx = Mx / 2 + 1, hz = Mz / 2 + 1;
        for (int i = threadIdx.x; i < KT * Mx; i += blockDim.x) {
            int c = i >> lgMx, kx = i & (Mx - 1);
            int col = c0 + c, ky = col >> lgMz, kz = col & (Mz - 1);
            T h = H[(int64_t(fold_index(ky, My)) * hz + fold_index(kz, Mz)) * hx + fold_index(kx, Mx)];
            s[c * pitch + kx] = cscale(s[c * pitch + kx], h);
        }
        __syncthreads();
        fft_lines<T>(s, Mx, KT, pitch, 1, tw_x, true, false);
    }
    for (int i = threadIdx.x; i < KT * nx_out; i += blockDim.x) {
        int x = i >> lgKT, c = i & (KT - 1);
        base[int64_t(x) * ncols + c] = s[c * pitch + x];
    }
}

constexpr int FFT_MAX_ELEMS = FFT_E * 512;   // one CTA (512 threads) per plane / pencil tile

inline int fft_threads(int elems) {
    int t = (elems + FFT_E - 1) / FFT_E;
    t = (t + 31) / 32 * 32;
    return t < 64 ? 64 : t;
}

}  // namespace sie

// ---------------------------------------------------------------------------
// Four-step FFT with the short DFTs in registers.
//
// For M = N1 N2, n = j2 + N2 j1 and k = k1 + N1 k2:
//   X[k1 + N1 k2] = sum_j2 W_N2^(j2 k2) W_M^(j2 k1) sum_j1 W_N1^(j1 k1) x[j2 + N2 j1]
// so a thread owning one j2 does a length-N1 DFT, multiplies by W_M^(j2 k1)
// and passes its N1 values through shared memory to the thread owning k1,
// which does a length-N2 DFT.  The inverse runs the same two steps in the
// opposite order: x[p2 + N2 p1] = sum_k1 W_N1^-(p1 k1) W_M^-(p2 k1)
// sum_k2 W_N2^-(p2 k2) X[k1 + N1 k2].  With the input zero beyond M/2 only
// j1 < N1/2 is loaded; with the output cropped to M/2 only p1 < N1/2 is stored.

namespace sie {

constexpr int FFT_NMAX = 16;                       // longest in-register DFT of the plane passes
// cos and sin of 2 pi i / 16, i = 0..7 (cos pi/8 = 0.9238..., sin pi/8 = 0.3826...)
__host__ __device__ constexpr double c16(int i) {
    return i == 0 ? 1.0 : i == 1 ? 0.92387953251128674 : i == 2 ? 0.70710678118654752 : i == 3 ? 0.38268343236508977
         : i == 4 ? 0.0 : i == 5 ? -0.38268343236508977 : i == 6 ? -0.70710678118654752 : -0.92387953251128674;
}
__host__ __device__ constexpr double s16(int i) {
    return i == 0 ? 0.0 : i == 1 ? 0.38268343236508977 : i == 2 ? 0.70710678118654752 : i == 3 ? 0.92387953251128674
         : i == 4 ? 1.0 : i == 5 ? 0.92387953251128674 : i == 6 ? 0.70710678118654752 : 0.38268343236508977;
}

// cos and sin of 2 pi t / 32 for odd t in [1, 16) (pi/16 and 3 pi/16 and their
// reflections: cos(pi/16) = 0.98078..., sin(pi/16) = 0.19509...,
// cos(3 pi/16) = 0.83146..., sin(3 pi/16) = 0.55557...).
__host__ __device__ constexpr double c32(int t) {
    return t == 1 ? 0.98078528040323045 : t == 3 ? 0.83146961230254524 : t == 5 ? 0.55557023301960222
         : t == 7 ? 0.19509032201612827 : t == 9 ? -0.19509032201612827 : t == 11 ? -0.55557023301960222
         : t == 13 ? -0.83146961230254524 : -0.98078528040323045;
}
__host__ __device__ constexpr double s32(int t) {
    return t == 1 ? 0.19509032201612827 : t == 3 ? 0.55557023301960222 : t == 5 ? 0.83146961230254524
         : t == 7 ? 0.98078528040323045 : t == 9 ? 0.98078528040323045 : t == 11 ? 0.83146961230254524
         : t == 13 ? 0.55557023301960222 : 0.19509032201612827;
}

// In-register DFTs of length 2, 4, 8, 16 and 32, natural order in and out,
// built from radix-4 (and one radix-2) butterflies with the twiddles as
// immediates; the direction is a compile-time choice.  DFT8 = 2 x 4 and
// DFT16 = 4 x 4 are four-step products in registers: the inner DFTs run over
// n = j + A m, the twiddle is W_N^(j k1) and the outer DFTs run over j; the
// final transposition is a register renaming.

// v * W_16^t, t in [0, 16): W_16^(t + 8) = -W_16^t, W_16^4 = -i (forward).
template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle_mul(C<T> b, int t) {
    C<T> r;
    const bool neg = t >= 8;
    t &= 7;
    if (t == 0) {
        r = b;
    } else if (t == 4) {
        if (INV) { r.x = -b.y; r.y = b.x; } else { r.x = b.y; r.y = -b.x; }
    } else {
        const T c = T(c16(t)), sn = INV ? T(s16(t)) : T(-s16(t));
        r.x = b.x * c - b.y * sn;
        r.y = b.x * sn + b.y * c;
    }
    if (neg) { r.x = -r.x; r.y = -r.y; }
    return r;
}

template <typename T, bool INV>
__device__ __forceinline__ void bfly4(C<T> &a0, C<T> &a1, C<T> &a2, C<T> &a3) {
    const C<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    C<T> t3;                          // -i d (forward), +i d (inverse)
    if (INV) { t3.x = -d.y; t3.y = d.x; } else { t3.x = d.y; t3.y = -d.x; }
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// v * W_32^t, t in [0, 16) (even t are the W_16 twiddles).
template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle32(C<T> b, int t) {
    if ((t & 1) == 0) return twiddle_mul<T, INV>(b, t >> 1);
    const T c = T(c32(t)), sn = INV ? T(s32(t)) : T(-s32(t));
    C<T> r;
    r.x = b.x * c - b.y * sn;
    r.y = b.x * sn + b.y * c;
    return r;
}

template <typename T, int N, bool INV, int NA>
__device__ __forceinline__ void dft_reg(C<T> (&v)[NA]) {
    static_assert(NA >= N, "register array shorter than the DFT");
    if constexpr (N == 32) {
        // n = j + 2m: DFT16 over m for j = 0, 1; twiddle W_32^(j k1); DFT2 over j
        C<T> a[16], b[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            a[m] = v[2 * m];
            b[m] = v[2 * m + 1];
        }
        dft_reg<T, 16, INV>(a);
        dft_reg<T, 16, INV>(b);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            const C<T> t = twiddle32<T, INV>(b[k1], k1);
            v[k1] = cadd(a[k1], t);
            v[k1 + 16] = csub(a[k1], t);
        }
    } else if constexpr (N == 2) {
        const C<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (N == 4) {
        bfly4<T, INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (N == 8) {
        // n = j + 2m: DFT4 over m for j = 0, 1; twiddle W_8^(j k1) = W_16^(2 j k1); DFT2 over j
        bfly4<T, INV>(v[0], v[2], v[4], v[6]);
        bfly4<T, INV>(v[1], v[3], v[5], v[7]);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[1 + 2 * k1] = twiddle_mul<T, INV>(v[1 + 2 * k1], 2 * k1);
        C<T> o[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {      // X[k1 + 4 k2], k2 = 0, 1
            o[k1] = cadd(v[2 * k1], v[2 * k1 + 1]);
            o[k1 + 4] = csub(v[2 * k1], v[2 * k1 + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = o[i];
    } else {
        static_assert(N == 16, "DFT length");
        // n = j + 4m: DFT4 over m for j = 0..3; twiddle W_16^(j k1); DFT4 over j
#pragma unroll
        for (int j = 0; j < 4; ++j) bfly4<T, INV>(v[j], v[j + 4], v[j + 8], v[j + 12]);
#pragma unroll
        for (int j = 1; j < 4; ++j)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) v[j + 4 * k1] = twiddle_mul<T, INV>(v[j + 4 * k1], j * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) bfly4<T, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
        C<T> o[16];                            // v[4 k1 + k2] = X[k1 + 4 k2]
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
}

// M -> (N1, N2): 8 = 2x4, 16 = 4x4, 32 = 4x8, 64 = 8x8, 128 = 8x16, 256 = 16x16
inline void split4(int M, int &N1, int &N2) {
    int lg = 0;
    while ((1 << lg) < M) ++lg;
    N1 = 1 << (lg / 2);
    N2 = M / N1;
}

// Calls BODY with compile-time (N1, N2) for the transform length M.
#define SIE_SPLIT_DISPATCH(M, BODY)                                        \
    switch (M) {                                                           \
        case 8: { constexpr int N1 = 2, N2 = 4; BODY; } break;             \
        case 16: { constexpr int N1 = 4, N2 = 4; BODY; } break;            \
        case 32: { constexpr int N1 = 4, N2 = 8; BODY; } break;            \
        case 64: { constexpr int N1 = 8, N2 = 8; BODY; } break;            \
        case 128: { constexpr int N1 = 8, N2 = 16; BODY; } break;          \
        default: { constexpr int N1 = 16, N2 = 16; BODY; } break;          \
    }

// The same for the pencil kernels, which also take M = 512 = 16 x 32.
#define SIE_SPLIT_DISPATCH_P(M, BODY)                                      \
    switch (M) {                                                           \
        case 8: { constexpr int N1 = 2, N2 = 4; BODY; } break;             \
        case 16: { constexpr int N1 = 4, N2 = 4; BODY; } break;            \
        case 32: { constexpr int N1 = 4, N2 = 8; BODY; } break;            \
        case 64: { constexpr int N1 = 8, N2 = 8; BODY; } break;            \
        case 128: { constexpr int N1 = 8, N2 = 16; BODY; } break;          \
        case 256: { constexpr int N1 = 16, N2 = 16; BODY; } break;         \
        default: { constexpr int N1 = 16, N2 = 32; BODY; } break;          \
    }

// Columns per pencil CTA: 16, or 8 when one factor is 32 (256 threads).
template <int N1, int N2> struct Pencil {
    static constexpr int NM = N1 > N2 ? N1 : N2;
    static constexpr int KT = NM > 16 ? 8 : 16;
    static constexpr int LGKT = KT == 16 ? 4 : 3;
    static constexpr int threads = KT * NM;
};

// Four-step twiddle tables of an axis of length M = N1 N2 (built at plan
// creation): tf[j2 * N1 + k1] = W_M^(j2 k1) for the forward pass 1 and
// ti[k1 * N2 + p2] = W_M^(k1 p2) for the inverse pass A (used conjugated).

// ---- x pencils.  Buffers [batch][rows][ncols], row x at x * ncols; one CTA
// per (batch, KT consecutive columns), KT * max(N1, N2) threads, a shared
// line per column (pitch M + 1).  The same kernels run the y pencils of
// grids whose (y, z) plane does not fit one CTA (batch = grid and
// x-frequency, rows = y, columns = z).

// Forward: in [batch][M/2][ncols] (zero-padded to M) -> out [batch][M][ncols].
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(256) k_fft_xf(const C<T> *__restrict__ in, C<T> *__restrict__ out, int ncols,
                                                const C<T> *__restrict__ tf) {
    constexpr int KT = Pencil<N1, N2>::KT, M = N1 * N2, pitch = M + 1, H1 = N1 / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *S = reinterpret_cast<C<T> *>(smem_raw);
    const int tiles = ncols / KT;
    const int b = blockIdx.x / tiles, c0 = (blockIdx.x % tiles) * KT;
    const int line = threadIdx.x & (KT - 1), q = threadIdx.x >> Pencil<N1, N2>::LGKT;
    C<T> *Sl = S + line * pitch;
    const int64_t stride = int64_t(N2) * ncols;
    C<T> v[Pencil<N1, N2>::NM];
    if (q < N2) {                      // pass 1: j2 = q, DFT over j1 (x = j2 + N2 j1 < M/2)
        const int j2 = q;
        const C<T> *src = in + int64_t(b) * (M / 2) * ncols + c0 + line + int64_t(j2) * ncols;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = j1 < H1 ? src[j1 * stride] : mk<T>(T(0), T(0));
        dft_reg<T, N1, false>(v);
        const C<T> *t = tf + j2 * N1;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Sl[k1 * N2 + j2] = k1 ? cmul(v[k1], t[k1]) : v[0];
    }
    __syncthreads();
    if (q < N1) {                      // pass 2: k1 = q, DFT over j2 -> X[k1 + N1 k2]
        const int k1 = q;
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = Sl[k1 * N2 + j2];
        dft_reg<T, N2, false>(v);
        C<T> *dst = out + int64_t(b) * M * ncols + c0 + line + int64_t(k1) * ncols;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) dst[N1 * k2 * int64_t(ncols)] = v[k2];
    }
}

// Inverse: in [batch][M][ncols] -> out [batch][M/2][ncols] (rows x < M/2 kept).
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(256) k_fft_xi(const C<T> *__restrict__ in, C<T> *__restrict__ out, int ncols,
                                                const C<T> *__restrict__ ti) {
    constexpr int KT = Pencil<N1, N2>::KT, M = N1 * N2, pitch = M + 1, H1 = N1 / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *S = reinterpret_cast<C<T> *>(smem_raw);
    const int tiles = ncols / KT;
    const int b = blockIdx.x / tiles, c0 = (blockIdx.x % tiles) * KT;
    const int line = threadIdx.x & (KT - 1), q = threadIdx.x >> Pencil<N1, N2>::LGKT;
    C<T> *Sl = S + line * pitch;
    C<T> v[Pencil<N1, N2>::NM];
    if (q < N1) {                      // pass A: k1 = q, inverse DFT over k2, conj twiddle
        const int k1 = q;
        const C<T> *src = in + int64_t(b) * M * ncols + c0 + line + int64_t(k1) * ncols;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = src[N1 * k2 * int64_t(ncols)];
        dft_reg<T, N2, true>(v);
        const C<T> *t = ti + k1 * N2;
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) {
            C<T> r = v[p2];
            if (p2) {
                const C<T> w = t[p2];
                r.x = v[p2].x * w.x + v[p2].y * w.y;
                r.y = v[p2].y * w.x - v[p2].x * w.y;
            }
            Sl[p2 * N1 + k1] = r;
        }
    }
    __syncthreads();
    if (q < N2) {                      // pass B: p2 = q, inverse DFT over k1, x = p2 + N2 p1 < M/2
        const int p2 = q;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = Sl[p2 * N1 + k1];
        dft_reg<T, N1, true>(v);
        C<T> *dst = out + int64_t(b) * (M / 2) * ncols + c0 + line + int64_t(p2) * ncols;
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) dst[p1 * int64_t(N2) * ncols] = v[p1];
    }
}

// ---- z rows of grids whose (y, z) plane does not fit one CTA.  After the x
// and y pencils the buffer holds rows [grid][kx][ky][z < N_z]; per row the
// zero-padded forward transform along z, the product with the kernel spectrum
// Hp[fold kx][fold ky][fold kz] (real, or complex for the lossy kernel) and
// the inverse transform cropped to z < N_z, in place.  RPC rows per CTA are
// staged in shared memory (pitch M_z + 1) with coalesced loads; the four-step
// passes map consecutive threads to consecutive rows, so every shared access
// of a warp hits distinct banks.
template <typename T>
__device__ __forceinline__ C<T> kernel_mul(C<T> v, T h) { return cscale(v, h); }
template <typename T>
__device__ __forceinline__ C<T> kernel_mul(C<T> v, C<T> h) { return cmul(v, h); }

template <int N1, int N2> struct ZRows {
    static constexpr int NM = N1 > N2 ? N1 : N2;
    static constexpr int RPC = 256 / NM;          // rows per CTA (256 threads)
    static constexpr int pitch = N1 * N2 + 1;
};

// Htab / gslot (both NULL for one spectrum Hp shared by every grid): grid g of
// the buffer uses the spectrum Htab[gslot[g]] (the lossy kernel, one spectrum
// per angular frequency of the grid's right-hand side).
template <typename T, int N1, int N2, typename HT>
__global__ void __launch_bounds__(256) k_fft_zconv(C<T> *__restrict__ buf, int lgMx, int lgMy,
                                                   const HT *__restrict__ Hp, const C<T> *__restrict__ tf,
                                                   const C<T> *__restrict__ ti, const HT *const *__restrict__ Htab,
                                                   const int32_t *__restrict__ gslot) {
    constexpr int Mz = N1 * N2, Nz = Mz / 2, H1 = N1 / 2, RPC = ZRows<N1, N2>::RPC, pitch = ZRows<N1, N2>::pitch;
    constexpr int LGNZ = Nz == 4 ? 2 : Nz == 8 ? 3 : Nz == 16 ? 4 : Nz == 32 ? 5 : Nz == 64 ? 6 : Nz == 128 ? 7 : 8;
    static_assert((1 << LGNZ) == Nz, "row length");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *S = reinterpret_cast<C<T> *>(smem_raw);
    const int64_t row0 = int64_t(blockIdx.x) * RPC;
    C<T> *g = buf + row0 * Nz;
    for (int i = threadIdx.x; i < RPC * Nz; i += blockDim.x) S[(i >> LGNZ) * pitch + (i & (Nz - 1))] = g[i];
    __syncthreads();
    const int r = threadIdx.x % RPC, q = threadIdx.x / RPC;
    C<T> *Sr = S + r * pitch;
    C<T> v[ZRows<N1, N2>::NM];
    if (q < N2) {                      // forward pass 1: j2 = q, DFT over j1 (z = j2 + N2 j1 < N_z)
        const int j2 = q;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = j1 < H1 ? Sr[j2 + N2 * j1] : mk<T>(T(0), T(0));
        dft_reg<T, N1, false>(v);
        const C<T> *t = tf + j2 * N1;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Sr[k1 * N2 + j2] = k1 ? cmul(v[k1], t[k1]) : v[0];
    }
    __syncthreads();
    const int k1 = q;
    if (q < N1) {                      // forward pass 2, kernel product, inverse pass A (in registers)
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = Sr[k1 * N2 + j2];
        dft_reg<T, N2, false>(v);      // v[k2] = X[k1 + N1 k2]
        const int Mx = 1 << lgMx, My = 1 << lgMy;
        const int64_t row = row0 + r;
        const int ky = int(row & (My - 1)), kx = int((row >> lgMy) & (Mx - 1));
        const HT *Hg = Htab ? Htab[gslot[row >> (lgMx + lgMy)]] : Hp;
        const HT *Hr = Hg + (int64_t(fold_index(kx, Mx)) * (My / 2 + 1) + fold_index(ky, My)) * (Mz / 2 + 1);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = kernel_mul<T>(v[k2], Hr[fold_index(k1 + N1 * k2, Mz)]);
        dft_reg<T, N2, true>(v);
    }
    __syncthreads();                   // every thread has read its pass-2 slots
    if (q < N1) {
        const C<T> *t = ti + k1 * N2;
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) {
            C<T> o = v[p2];
            if (p2) {
                const C<T> w = t[p2];
                o.x = v[p2].x * w.x + v[p2].y * w.y;
                o.y = v[p2].y * w.x - v[p2].x * w.y;
            }
            Sr[p2 * N1 + k1] = o;
        }
    }
    __syncthreads();
    const int p2 = q;
    if (q < N2) {                      // inverse pass B: p2 = q, DFT over k1, z = p2 + N2 p1 < N_z
#pragma unroll
        for (int kk = 0; kk < N1; ++kk) v[kk] = Sr[p2 * N1 + kk];
        dft_reg<T, N1, true>(v);
    }
    __syncthreads();                   // every thread has read its pass-B slots
    if (q < N2) {
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) Sr[p2 + N2 * p1] = v[p1];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RPC * Nz; i += blockDim.x) g[i] = S[(i >> LGNZ) * pitch + (i & (Nz - 1))];
}

// Forward FFT of contiguous full rows of length M in place (the kernel
// spectrum at plan creation when the (y, z) plane does not fit one CTA):
// rows_per_cta * M <= FFT_E * blockDim.x elements staged per CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_rows(C<T> *__restrict__ buf, int M, int rows_per_cta,
                                                  const C<T> *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *s = reinterpret_cast<C<T> *>(smem_raw);
    C<T> *g = buf + int64_t(blockIdx.x) * rows_per_cta * M;
    const int n = rows_per_cta * M;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[i] = g[i];
    __syncthreads();
    fft_lines<T>(s, M, rows_per_cta, M, 1, tw, false, false);
    for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = s[i];
}

// ---- (y, z) plane passes with compile-time split (see k_fft_yzc).  The
// input extent is half of each padded length (Ny = My/2, Nz = Mz/2).
template <typename T, int N1, int N2>   // F1: z pass 1, rows y < Ny, global -> P row slots
__device__ __forceinline__ void yz_f1(const C<T> *in, C<T> *P, int pitch, int Ny, const C<T> *tfz) {
    constexpr int Mz = N1 * N2, Nz = Mz / 2, H1 = N1 / 2;
    constexpr int LG2 = N2 == 2 ? 1 : N2 == 4 ? 2 : N2 == 8 ? 3 : 4;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N2; it += blockDim.x) {
        const int y = it >> LG2, j2 = it & (N2 - 1);
        const C<T> *src = in + y * Nz + j2;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = j1 < H1 ? src[N2 * j1] : mk<T>(T(0), T(0));
        dft_reg<T, N1, false>(v);
        const C<T> *t = tfz + j2 * N1;
        C<T> *row = P + y * pitch + j2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) row[k1 * N2] = k1 ? cmul(v[k1], t[k1]) : v[0];
    }
}
template <typename T, int N1, int N2>   // F2: z pass 2, P row slots -> Q natural rows
__device__ __forceinline__ void yz_f2(const C<T> *P, C<T> *Q, int pitch, int lgNy) {
    C<T> v[FFT_NMAX];
    const int Ny = 1 << lgNy;
    for (int it = threadIdx.x; it < Ny * N1; it += blockDim.x) {
        const int y = it & (Ny - 1), k1 = it >> lgNy;
        const C<T> *row = P + y * pitch + k1 * N2;
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = row[j2];
        dft_reg<T, N2, false>(v);
        C<T> *out = Q + y * pitch + k1;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) out[N1 * k2] = v[k2];
    }
}
template <typename T, int N1, int N2>   // F3: y pass 1, all columns, Q rows < Ny -> P column slots
__device__ __forceinline__ void yz_f3(const C<T> *Q, C<T> *P, int pitch, int lgMz, const C<T> *tfy) {
    constexpr int H1 = N1 / 2;
    C<T> v[FFT_NMAX];
    const int Mz = 1 << lgMz;
    for (int it = threadIdx.x; it < Mz * N2; it += blockDim.x) {
        const int kz = it & (Mz - 1), j2 = it >> lgMz;
        const C<T> *col = Q + j2 * pitch + kz;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = j1 < H1 ? col[N2 * j1 * pitch] : mk<T>(T(0), T(0));
        dft_reg<T, N1, false>(v);
        const C<T> *t = tfy + j2 * N1;
        C<T> *o = P + j2 * pitch + kz;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) o[k1 * N2 * pitch] = k1 ? cmul(v[k1], t[k1]) : v[0];
    }
}
template <typename T, int N1, int N2>   // I2: y inverse pass B, P -> Q rows y < Ny
__device__ __forceinline__ void yz_i2(const C<T> *P, C<T> *Q, int pitch, int lgMz) {
    constexpr int H1 = N1 / 2;
    C<T> v[FFT_NMAX];
    const int Mz = 1 << lgMz;
    for (int it = threadIdx.x; it < Mz * N2; it += blockDim.x) {
        const int kz = it & (Mz - 1), p2 = it >> lgMz;
        const C<T> *src = P + p2 * N1 * pitch + kz;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[k1 * pitch];
        dft_reg<T, N1, true>(v);
        C<T> *o = Q + p2 * pitch + kz;
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) o[N2 * p1 * pitch] = v[p1];
    }
}
// I3 writes row slot p2 + N2 k1 (not k1 + N1 p2) so that I4's threads, which
// run over p2 with k1 fixed per load, read consecutive slots: both passes hit
// distinct shared-memory banks.
template <typename T, int N1, int N2>   // I3: z inverse pass A, Q rows -> P row slots
__device__ __forceinline__ void yz_i3(const C<T> *Q, C<T> *P, int pitch, int lgNy, const C<T> *tiz) {
    C<T> v[FFT_NMAX];
    const int Ny = 1 << lgNy;
    for (int it = threadIdx.x; it < Ny * N1; it += blockDim.x) {
        const int y = it & (Ny - 1), k1 = it >> lgNy;
        const C<T> *src = Q + y * pitch + k1;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = src[N1 * k2];
        dft_reg<T, N2, true>(v);
        const C<T> *t = tiz + k1 * N2;
        C<T> *o = P + y * pitch + k1 * N2;
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) {
            C<T> r = v[p2];
            if (p2) {
                const C<T> w = t[p2];
                r.x = v[p2].x * w.x + v[p2].y * w.y;
                r.y = v[p2].y * w.x - v[p2].x * w.y;
            }
            o[p2] = r;
        }
    }
}
template <typename T, int N1, int N2>   // I4: z inverse pass B, P row slots -> global, z < Nz
__device__ __forceinline__ void yz_i4(const C<T> *P, C<T> *out, int pitch, int Ny) {
    constexpr int Mz = N1 * N2, Nz = Mz / 2, H1 = N1 / 2;
    constexpr int LG2 = N2 == 2 ? 1 : N2 == 4 ? 2 : N2 == 8 ? 3 : 4;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N2; it += blockDim.x) {
        const int y = it >> LG2, p2 = it & (N2 - 1);
        const C<T> *src = P + y * pitch + p2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = src[k1 * N2];
        dft_reg<T, N1, true>(v);
        C<T> *o = out + y * Nz + p2;
#pragma unroll
        for (int p1 = 0; p1 < H1; ++p1) o[N2 * p1] = v[p1];
    }
}

// y pass 2, times H(kx, ky, kz), inverse y pass A, in place on the column
// slots of P (rows k1 N2 + j2 in, rows k1 + N1 p2 out).  A round takes
// CW = blockDim / N1 complete kz columns (every k1 of them), so all reads of a
// column precede all writes to it; lanes run over kz (conflict-free).
// Hk: this kx's kernel spectrum [fold(ky)][fold(kz)], pitch Mz/2 + 1.
// v times a kernel value: real (static kernel) or complex (lossy kernel).
template <typename T> __device__ __forceinline__ C<T> hmul(C<T> v, T h) { return cscale(v, h); }
template <typename T> __device__ __forceinline__ C<T> hmul(C<T> v, C<T> h) { return cmul(v, h); }

template <typename T, int N1, int N2, typename HT>
__device__ __forceinline__ void yz_mid(C<T> *P, int pitch, int lgMz, const HT *__restrict__ Hk,
                                       const C<T> *__restrict__ tiy) {
    constexpr int My = N1 * N2;
    const int Mz = 1 << lgMz, hz = Mz / 2 + 1;
    const int CW = blockDim.x / N1;
    const int k1 = threadIdx.x / CW, kzl = threadIdx.x - k1 * CW;
    C<T> v[FFT_NMAX];
    for (int kz0 = 0; kz0 < Mz; kz0 += CW) {
        const int kz = kz0 + kzl;
        const bool act = k1 < N1 && kz < Mz;
        if (act) {
            const C<T> *col = P + k1 * N2 * pitch + kz;
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) v[j2] = col[j2 * pitch];
            dft_reg<T, N2, false>(v);      // v[k2] = X[ky = k1 + N1 k2]
            const HT *h = Hk + fold_index(kz, Mz);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) v[k2] = hmul<T>(v[k2], h[fold_index(k1 + N1 * k2, My) * hz]);
            dft_reg<T, N2, true>(v);
            const C<T> *t = tiy + k1 * N2;
#pragma unroll
            for (int p2 = 1; p2 < N2; ++p2) {
                const C<T> w = t[p2];
                C<T> r;
                r.x = v[p2].x * w.x + v[p2].y * w.y;   // times conj(w)
                r.y = v[p2].y * w.x - v[p2].x * w.y;
                v[p2] = r;
            }
        }
        __syncthreads();
        if (act) {
            C<T> *o = P + k1 * pitch + kz;
#pragma unroll
            for (int p2 = 0; p2 < N2; ++p2) o[p2 * N1 * pitch] = v[p2];
        }
        __syncthreads();
    }
}

// The (y, z) part of the 3-D convolution for one x-frequency plane, in place:
// plane [Ny][Nz] of buffer [batch][Mx][Ny][Nz] -> zero-padded 2-D FFT ->
// times H(kx, ., .) -> inverse 2-D FFT -> cropped to [Ny][Nz].  Four-step in
// both axes through two shared buffers (P: My x pitch, Q: Ny x pitch) so that
// every step reads one and writes the other.  One CTA per (batch, kx), NT
// threads (512 in FP32: two CTAs and 32 warps per SM; 256 in FP64, whose
// plane fills the shared memory of one SM).
// Hp: kernel spectrum [fold(kx)][fold(ky)][fold(kz)], scaled by 1/(Mx My Mz):
// real (HT = T, the static kernel) or complex (HT = C<T>, the lossy kernel).
// Htab / gslot: as in k_fft_zconv (grid g = blockIdx.x / Mx uses Htab[gslot[g]]).
template <typename T, int NT, typename HT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_fft_yzc(C<T> *__restrict__ buf, int lgMx, int My, int Mz,
                                                 const HT *__restrict__ Hp, const C<T> *__restrict__ tfy,
                                                 const C<T> *__restrict__ tiy, const C<T> *__restrict__ tfz,
                                                 const C<T> *__restrict__ tiz, const HT *const *__restrict__ Htab,
                                                 const int32_t *__restrict__ gslot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pitch = Mz + 1, Ny = My / 2, Nz = Mz / 2;
    const int lgNy = ilog2(Ny), lgMz = ilog2(Mz);
    const int Mx = 1 << lgMx;
    const int kx = blockIdx.x & (Mx - 1);
    C<T> *P = reinterpret_cast<C<T> *>(smem_raw);
    C<T> *Qb = P + My * pitch;
    C<T> *plane = buf + int64_t(blockIdx.x) * Ny * Nz;
    const HT *Hg = Htab ? Htab[gslot[blockIdx.x >> lgMx]] : Hp;
    const HT *Hk = Hg + int64_t(fold_index(kx, Mx)) * (My / 2 + 1) * (Mz / 2 + 1);
    SIE_SPLIT_DISPATCH(Mz, (yz_f1<T, N1, N2>(plane, P, pitch, Ny, tfz)));
    __syncthreads();
    SIE_SPLIT_DISPATCH(Mz, (yz_f2<T, N1, N2>(P, Qb, pitch, lgNy)));
    __syncthreads();
    SIE_SPLIT_DISPATCH(My, (yz_f3<T, N1, N2>(Qb, P, pitch, lgMz, tfy)));
    __syncthreads();
    SIE_SPLIT_DISPATCH(My, (yz_mid<T, N1, N2, HT>(P, pitch, lgMz, Hk, tiy)));
    SIE_SPLIT_DISPATCH(My, (yz_i2<T, N1, N2>(P, Qb, pitch, lgMz)));
    __syncthreads();
    SIE_SPLIT_DISPATCH(Mz, (yz_i3<T, N1, N2>(Qb, P, pitch, lgNy, tiz)));
    __syncthreads();
    SIE_SPLIT_DISPATCH(Mz, (yz_i4<T, N1, N2>(P, plane, pitch, Ny)));
}

}  // namespace sie
