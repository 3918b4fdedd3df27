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
