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

constexpr int FFT_NMAX = 16;                       // longest in-register DFT
// cos and sin of 2 pi i / 16, i = 0..7 (cos pi/8 = 0.9238..., sin pi/8 = 0.3826...)
__host__ __device__ constexpr double c16(int i) {
    return i == 0 ? 1.0 : i == 1 ? 0.92387953251128674 : i == 2 ? 0.70710678118654752 : i == 3 ? 0.38268343236508977
         : i == 4 ? 0.0 : i == 5 ? -0.38268343236508977 : i == 6 ? -0.70710678118654752 : -0.92387953251128674;
}
__host__ __device__ constexpr double s16(int i) {
    return i == 0 ? 0.0 : i == 1 ? 0.38268343236508977 : i == 2 ? 0.70710678118654752 : i == 3 ? 0.92387953251128674
         : i == 4 ? 1.0 : i == 5 ? 0.92387953251128674 : i == 6 ? 0.70710678118654752 : 0.38268343236508977;
}

// In-register DFT of v[0..N), N a power of two <= 16: bit reversal, then
// radix-2 butterflies with twiddles W_len^j = exp(-+ 2 pi i j / len), the
// direction a compile-time choice so twiddles are immediates; multiplications
// by 1 and by -+i are done as moves.
template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle_mul(C<T> b, int ti) {
    C<T> t;
    if (ti == 0) return b;
    if (ti == 4) {                      // W_16^4 = -i (forward), +i (inverse)
        if (INV) { t.x = -b.y; t.y = b.x; } else { t.x = b.y; t.y = -b.x; }
        return t;
    }
    const T c = T(c16(ti)), sn = INV ? T(s16(ti)) : T(-s16(ti));
    t.x = b.x * c - b.y * sn;
    t.y = b.x * sn + b.y * c;
    return t;
}

template <typename T, int N, bool INV>
__device__ __forceinline__ void dft_reg(C<T> (&v)[FFT_NMAX]) {
    constexpr int LG = N == 2 ? 1 : N == 4 ? 2 : N == 8 ? 3 : 4;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 0; b < LG; ++b) r |= ((i >> b) & 1) << (LG - 1 - b);
        if (r > i) { C<T> t = v[i]; v[i] = v[r]; v[r] = t; }
    }
#pragma unroll
    for (int st = 0; st < LG; ++st) {
        const int len = 2 << st, half = 1 << st;
#pragma unroll
        for (int s = 0; s < N; s += len) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const C<T> t = twiddle_mul<T, INV>(v[s + j + half], j * (16 / len));
                v[s + j + half] = csub(v[s + j], t);
                v[s + j] = cadd(v[s + j], t);
            }
        }
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

template <typename T, int N1, int N2>
__device__ __forceinline__ void x4_body(C<T> *S, C<T> *base, int ncols, int nx, int My, int Mz, int c0,
                                        const C<T> *__restrict__ tw, const T *__restrict__ H) {
    constexpr int KT = 16, Mx = N1 * N2, pitch = Mx + 1;
    const int line = threadIdx.x & (KT - 1), q = threadIdx.x >> 4;
    C<T> *Sl = S + line * pitch;
    const C<T> zero = mk<T>(T(0), T(0));
    C<T> v[FFT_NMAX];
    if (q < N2) {                      // pass 1: j2 = q, DFT over j1 (input zero for x >= nx)
        const int j2 = q;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) {
            const int x = j2 + N2 * j1;
            v[j1] = x < nx ? base[int64_t(x) * ncols + line] : zero;
        }
        dft_reg<T, N1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) Sl[k1 * N2 + j2] = k1 ? cmul(v[k1], tw[(j2 * k1) & (Mx - 1)]) : v[0];
    }
    __syncthreads();
    constexpr int hx = Mx / 2 + 1;
    const int hz = Mz / 2 + 1;
    const int col = c0 + line, ky = col / Mz, kz = col & (Mz - 1);
    const T *Hc = H + (int64_t(fold_index(ky, My)) * hz + fold_index(kz, Mz)) * hx;
    if (q < N1) {                      // pass 2: k1 = q, DFT over j2, times H, inverse DFT over k2
        const int k1 = q;
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = Sl[k1 * N2 + j2];
        dft_reg<T, N2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = cscale(v[k2], Hc[fold_index(k1 + N1 * k2, Mx)]);
        dft_reg<T, N2, true>(v);
#pragma unroll
        for (int p2 = 1; p2 < N2; ++p2) {
            C<T> w = tw[(p2 * k1) & (Mx - 1)];
            w.y = -w.y;
            v[p2] = cmul(v[p2], w);
        }
    }
    __syncthreads();                   // pass-2 reads complete before pass-A writes
    if (q < N1) {
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) Sl[p2 * N1 + q] = v[p2];
    }
    __syncthreads();
    if (q < N2) {                      // inverse pass B: p2 = q, DFT over k1, keep x < nx
        const int p2 = q;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = Sl[p2 * N1 + k1];
        dft_reg<T, N1, true>(v);
#pragma unroll
        for (int p1 = 0; p1 < N1; ++p1) {
            const int x = p2 + N2 * p1;
            if (x < nx) base[int64_t(x) * ncols + line] = v[p1];
        }
    }
}

// x-pencils, four-step: forward FFT, times H, inverse FFT (the middle pass of
// the 3-D convolution).  Buffer [batch][x][ncols]; one CTA per (batch, 16
// columns); 16 * max(N1, N2) threads.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x4(C<T> *__restrict__ buf, int64_t batch_stride, int ncols, int nx,
                                                int Mx, int My, int Mz, const C<T> *__restrict__ tw,
                                                const T *__restrict__ H) {
    constexpr int KT = 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *S = reinterpret_cast<C<T> *>(smem_raw);
    const int tiles = ncols / KT;
    const int b = blockIdx.x / tiles, c0 = (blockIdx.x % tiles) * KT;
    C<T> *base = buf + b * batch_stride + c0;
    SIE_SPLIT_DISPATCH(Mx, (x4_body<T, N1, N2>(S, base, ncols, nx, My, Mz, c0, tw, H)));
}

// ---- (y, z) plane passes with compile-time split (see k_fft_yz4)
template <typename T, int N1, int N2>   // F1: z pass 1, rows y < Ny, global -> P row slots
__device__ __forceinline__ void yz_f1(const C<T> *in, C<T> *P, int pitch, int Ny, int Nz, const C<T> *twz) {
    constexpr int Mz = N1 * N2;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N2; it += blockDim.x) {
        const int y = it / N2, j2 = it & (N2 - 1);
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) {
            const int z = j2 + N2 * j1;
            v[j1] = z < Nz ? in[y * Nz + z] : mk<T>(T(0), T(0));
        }
        dft_reg<T, N1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) P[y * pitch + k1 * N2 + j2] = k1 ? cmul(v[k1], twz[(j2 * k1) & (Mz - 1)]) : v[0];
    }
}
template <typename T, int N1, int N2>   // F2: z pass 2, P row slots -> Q natural rows
__device__ __forceinline__ void yz_f2(const C<T> *P, C<T> *Q, int pitch, int Ny) {
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N1; it += blockDim.x) {
        const int y = it % Ny, k1 = it / Ny;
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = P[y * pitch + k1 * N2 + j2];
        dft_reg<T, N2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) Q[y * pitch + k1 + N1 * k2] = v[k2];
    }
}
template <typename T, int N1, int N2>   // F3: y pass 1, all columns, Q rows < Ny -> P column slots
__device__ __forceinline__ void yz_f3(const C<T> *Q, C<T> *P, int pitch, int Ny, int Mz, const C<T> *twy) {
    constexpr int My = N1 * N2;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Mz * N2; it += blockDim.x) {
        const int kz = it % Mz, j2 = it / Mz;
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) {
            const int y = j2 + N2 * j1;
            v[j1] = y < Ny ? Q[y * pitch + kz] : mk<T>(T(0), T(0));
        }
        dft_reg<T, N1, false>(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1)
            P[(k1 * N2 + j2) * pitch + kz] = k1 ? cmul(v[k1], twy[(j2 * k1) & (My - 1)]) : v[0];
    }
}
template <typename T, int N1, int N2>   // F4: y pass 2, P column slots -> global spectrum
__device__ __forceinline__ void yz_f4(const C<T> *P, C<T> *out, int pitch, int Mz) {
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Mz * N1; it += blockDim.x) {
        const int kz = it % Mz, k1 = it / Mz;
#pragma unroll
        for (int j2 = 0; j2 < N2; ++j2) v[j2] = P[(k1 * N2 + j2) * pitch + kz];
        dft_reg<T, N2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) out[(k1 + N1 * k2) * Mz + kz] = v[k2];
    }
}
template <typename T, int N1, int N2>   // I1: y inverse pass A, global spectrum -> P
__device__ __forceinline__ void yz_i1(const C<T> *in, C<T> *P, int pitch, int Mz, const C<T> *twy) {
    constexpr int My = N1 * N2;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Mz * N1; it += blockDim.x) {
        const int kz = it % Mz, k1 = it / Mz;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = in[(k1 + N1 * k2) * Mz + kz];
        dft_reg<T, N2, true>(v);
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) {
            C<T> w = twy[(p2 * k1) & (My - 1)];
            w.y = -w.y;
            P[(p2 * N1 + k1) * pitch + kz] = (p2 && k1) ? cmul(v[p2], w) : v[p2];
        }
    }
}
template <typename T, int N1, int N2>   // I2: y inverse pass B, P -> Q rows y < Ny
__device__ __forceinline__ void yz_i2(const C<T> *P, C<T> *Q, int pitch, int Ny, int Mz) {
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Mz * N2; it += blockDim.x) {
        const int kz = it % Mz, p2 = it / Mz;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = P[(p2 * N1 + k1) * pitch + kz];
        dft_reg<T, N1, true>(v);
#pragma unroll
        for (int p1 = 0; p1 < N1; ++p1) {
            const int y = p2 + N2 * p1;
            if (y < Ny) Q[y * pitch + kz] = v[p1];
        }
    }
}
template <typename T, int N1, int N2>   // I3: z inverse pass A, Q rows -> P row slots
__device__ __forceinline__ void yz_i3(const C<T> *Q, C<T> *P, int pitch, int Ny, const C<T> *twz) {
    constexpr int Mz = N1 * N2;
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N1; it += blockDim.x) {
        const int y = it % Ny, k1 = it / Ny;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = Q[y * pitch + k1 + N1 * k2];
        dft_reg<T, N2, true>(v);
#pragma unroll
        for (int p2 = 0; p2 < N2; ++p2) {
            C<T> w = twz[(p2 * k1) & (Mz - 1)];
            w.y = -w.y;
            P[y * pitch + p2 * N1 + k1] = (p2 && k1) ? cmul(v[p2], w) : v[p2];
        }
    }
}
template <typename T, int N1, int N2>   // I4: z inverse pass B, P row slots -> global, z < Nz
__device__ __forceinline__ void yz_i4(const C<T> *P, C<T> *out, int pitch, int Ny, int Nz) {
    C<T> v[FFT_NMAX];
    for (int it = threadIdx.x; it < Ny * N2; it += blockDim.x) {
        const int y = it / N2, p2 = it & (N2 - 1);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = P[y * pitch + p2 * N1 + k1];
        dft_reg<T, N1, true>(v);
#pragma unroll
        for (int p1 = 0; p1 < N1; ++p1) {
            const int z = p2 + N2 * p1;
            if (z < Nz) out[y * Nz + z] = v[p1];
        }
    }
}

// (y, z) planes, four-step in both axes, two shared buffers (P: My x pitch,
// Q: Ny x pitch) so that every step reads one buffer and writes the other.
// Forward: input [Ny][Nz] (zero-padded), output the full [My][Mz] spectrum.
// Inverse: input [My][Mz], output [Ny][Nz].  One CTA per plane.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_yz4(const C<T> *__restrict__ src, int64_t src_stride,
                                                 C<T> *__restrict__ dst, int64_t dst_stride, int Ny, int Nz, int My,
                                                 int Mz, const C<T> *__restrict__ twy, const C<T> *__restrict__ twz,
                                                 int inverse) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pitch = Mz + 1;
    C<T> *P = reinterpret_cast<C<T> *>(smem_raw);
    C<T> *Qb = P + My * pitch;
    const C<T> *in = src + blockIdx.x * src_stride;
    C<T> *out = dst + blockIdx.x * dst_stride;
    if (!inverse) {
        SIE_SPLIT_DISPATCH(Mz, (yz_f1<T, N1, N2>(in, P, pitch, Ny, Nz, twz)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(Mz, (yz_f2<T, N1, N2>(P, Qb, pitch, Ny)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(My, (yz_f3<T, N1, N2>(Qb, P, pitch, Ny, Mz, twy)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(My, (yz_f4<T, N1, N2>(P, out, pitch, Mz)));
    } else {
        SIE_SPLIT_DISPATCH(My, (yz_i1<T, N1, N2>(in, P, pitch, Mz, twy)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(My, (yz_i2<T, N1, N2>(P, Qb, pitch, Ny, Mz)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(Mz, (yz_i3<T, N1, N2>(Qb, P, pitch, Ny, twz)));
        __syncthreads();
        SIE_SPLIT_DISPATCH(Mz, (yz_i4<T, N1, N2>(P, out, pitch, Ny, Nz)));
    }
}

}  // namespace sie
