// Block-cooperative complex FFTs held in registers, exchanged through shared memory.
//
// A transform of size P (a power of two, 2..4096) is owned by T = P/E threads of one CTA; thread
// t (0 <= t < T) holds the E elements with indices t + T*r, r = 0..E-1, in v[r]. That layout is
// both the input and the output layout, so pointwise work (chirps, spectra) happens in registers.
// The transform is a Stockham autosort decimation-in-time FFT: every pass reads radix-R groups
// at stride P/R straight from registers, applies the twiddles exp(dir*2*pi*i*s*k/(Ns*R)) from an
// FP64-built ladder table (consecutive k at consecutive addresses), does a radix-R DFT in registers, and scatters its R outputs to shared memory in
// Stockham order; after a barrier each thread reloads its E elements at stride T. R = E except for
// a final smaller pass when P is not a power of E. The exchange positions are XOR-swizzled per
// pass (xpos below) so that neither the scatter nor the gather serialises on shared-memory banks.
// The last pass needs no exchange: its Stockham positions are t + T*(q + Q*s), the thread's own
// slots, so its outputs stay in registers (a transform of p passes makes p - 1 exchanges).
//
// All threads of a group of T threads must call the same transform the same number of times;
// several groups may run independent transforms of the same size, each on its own shared buffer.
// The passes synchronise with __syncthreads() (bar = 0: all threads of the CTA call the transform)
// or, with bar = 1 + group index, only among the group's T threads (a named barrier, or a warp
// barrier when the group lies inside one warp), so groups do not wait for each other. Every call
// executes at least one such barrier, and its last shared-memory access precedes its last barrier,
// so the threads it synchronises may reuse the buffer (or any other shared memory they read before
// the call) right after it returns. Inverse transforms are not normalised: every 1/P factor is
// folded into the plan's tables.
#pragma once

#include "common.cuh"

namespace fbst {

// Shared-memory position of element i in the exchange of a pass with sub-transform size NS and
// radix R, for a transform of size P. The low 4 bits of the index (an 8-byte element's bank within
// a 128-byte row) are XORed with a key that is constant over every aligned run of 16 indices, so
// the gather (t + T*r, consecutive over threads) stays conflict-free, and that separates the
// groups of the scatter: the scatter of a pass writes base + s*NS with base = (j/NS)*NS*R + j%NS,
// i.e. groups of NS consecutive threads NS*R apart. For NS*R >= 16 the key (j/NS)*NS spreads the
// 16/NS groups of a half-warp over distinct banks; for NS*R < 16 (first passes, NS = 1) the row
// index i >> 4 does. The map permutes each aligned block of 16, so no padding is needed.
template <int P, int NS, int R>
__device__ __forceinline__ int xpos(int i) {
  if constexpr (P < 16) {
    return i;
  } else if constexpr (NS * R >= 16) {
    return i ^ (((i / (NS * R)) * NS) & 15);
  } else {
    return i ^ ((i >> 4) & 15);
  }
}

// Barrier of the transform's threads: the CTA (bar = 0) or the group of T threads that owns
// barrier id bar (T a multiple of 32), or its warp (T <= 32).
template <int T>
__device__ __forceinline__ void fft_sync(int bar) {
  if (bar == 0) {
    __syncthreads();
  } else if constexpr (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(T) : "memory");
  }
}

// Shared-memory elements one transform of size P needs.
template <typename V> constexpr int fft_smem_elems(int P) { return P; }

// cos(2*pi*j/16), j = 0..15, for the in-register butterflies.
__host__ __device__ constexpr double cos16(int j) {
  constexpr double c1 = 0.92387953251128675613, c2 = 0.70710678118654752440,
                   c3 = 0.38268343236508977173;
  switch (((j % 16) + 16) % 16) {
    case 0: return 1.0;   case 1: return c1;   case 2: return c2;   case 3: return c3;
    case 4: return 0.0;   case 5: return -c3;  case 6: return -c2;  case 7: return -c1;
    case 8: return -1.0;  case 9: return -c1;  case 10: return -c2; case 11: return -c3;
    case 12: return 0.0;  case 13: return c3;  case 14: return c2;  default: return c1;
  }
}

// a * exp(DIR*2*pi*i*K/R) for a compile-time root (R divides 16).
template <int R, int K, int DIR, typename V>
__device__ __forceinline__ V mul_root(V a) {
  constexpr int k = ((K % R) + R) % R;
  using S = decltype(a.x);
  if constexpr (k == 0) {
    return a;
  } else if constexpr (2 * k == R) {
    return V{-a.x, -a.y};
  } else if constexpr (4 * k == R) {
    return DIR < 0 ? V{a.y, -a.x} : V{-a.y, a.x};
  } else if constexpr (4 * k == 3 * R) {
    return DIR < 0 ? V{-a.y, a.x} : V{a.y, -a.x};
  } else {
    constexpr int j = k * (16 / R);
    constexpr S c = static_cast<S>(cos16(j));
    constexpr S s = static_cast<S>(DIR * cos16(j - 4));  // sin(2*pi*j/16) = cos(2*pi*(j-4)/16)
    return V{a.x * c - a.y * s, a.x * s + a.y * c};
  }
}

template <int R, int DIR, int K, typename V>
__device__ __forceinline__ void dft_combine(V* x, const V* e, const V* o) {
  if constexpr (K < R / 2) {
    const V t = mul_root<R, K, DIR>(o[K]);
    x[K] = cadd(e[K], t);
    x[K + R / 2] = csub(e[K], t);
    dft_combine<R, DIR, K + 1>(x, e, o);
  }
}

// In-register DFT of size R (1, 2, 4, 8 or 16): x[k] <- sum_n x[n] exp(DIR*2*pi*i*n*k/R).
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft(V* x) {
  if constexpr (R == 2) {
    const V a = x[0];
    x[0] = cadd(a, x[1]);
    x[1] = csub(a, x[1]);
  } else if constexpr (R > 2) {
    V e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    dft<R / 2, DIR>(e);
    dft<R / 2, DIR>(o);
    dft_combine<R, DIR, 0>(x, e, o);
  }
}

// One Stockham pass (current sub-transform size NS) followed by the remaining passes.
// v[f][r] is element t + T*r of transform f; sbuf holds NF consecutive buffers of P elements.
template <int P, int E, int NF, int DIR, int NS, typename V>
__device__ __forceinline__ void fft_passes(V (&v)[NF][E], V* sbuf, const V* __restrict__ tw, int t, int bar,
                                           int gkey) {
  if constexpr (NS < P) {
    constexpr int R = (P / NS < E) ? (P / NS) : E;
    constexpr int T = P / E;
    constexpr int Q = E / R;                       // butterflies per thread in this pass
    constexpr int SB = fft_smem_elems<V>(P);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = t + T * q;                     // butterfly index, 0 <= j < P/R
      const int k = j & (NS - 1);                  // position inside the current sub-transform
      V w[R];
      if constexpr (NS > 1) {
        // Load the powers w^1, w^2, w^4, w^8 of the pass twiddle and form the others as products
        // of at most three of them (L1 traffic of log2(R) loads instead of R-1).
#pragma unroll
        for (int s = 1; s < R; s <<= 1) {
          V ws = tw[(NS * R / s) / 2 - 1 + k];  // ladder entry k of M = NS*R/s: exp(-2*pi*i*s*k/(NS*R))
          if constexpr (DIR > 0) ws.y = -ws.y;
          w[s] = ws;
        }
#pragma unroll
        for (int s = 3; s < R; ++s) {
          if ((s & (s - 1)) != 0) {
            const int hi = 1 << (31 - __clz(s));
            w[s] = cmul(w[hi], w[s - hi]);
          }
        }
      }
      const int base = (j - k) * R + k;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        V x[R];
#pragma unroll
        for (int s = 0; s < R; ++s) x[s] = v[f][q + Q * s];
        if constexpr (NS > 1) {
#pragma unroll
          for (int s = 1; s < R; ++s) x[s] = cmul(x[s], w[s]);
        }
        dft<R, DIR>(x);
        if constexpr (NS * R == P) {
          // Last pass: output s lands at base + s*NS = t + T*(q + Q*s), this thread's slot q + Q*s.
#pragma unroll
          for (int s = 0; s < R; ++s) v[f][q + Q * s] = x[s];
        } else {
#pragma unroll
          for (int s = 0; s < R; ++s) sbuf[f * SB + (xpos<P, NS, R>(base + s * NS) ^ gkey)] = x[s];
        }
      }
    }
    if constexpr (NS * R == P) {
      if constexpr (NS == 1) fft_sync<T>(bar);  // single-pass transform: keep one barrier per call
    } else {
      fft_sync<T>(bar);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
#pragma unroll
        for (int r = 0; r < E; ++r) v[f][r] = sbuf[f * SB + (xpos<P, NS, R>(t + T * r) ^ gkey)];
      }
      fft_sync<T>(bar);
      fft_passes<P, E, NF, DIR, NS * R>(v, sbuf, tw, t, bar, gkey);
    }
  }
}

// NF simultaneous transforms of size P in the strided register layout described above.
// DIR = -1: forward (exp(-i...)); DIR = +1: unnormalised inverse. sbuf: NF*fft_smem_elems(P).
// bar: 0 for CTA-wide barriers, else 1 + the group index (1..15) of a group of P/E threads.
template <int P, int E, int NF, int DIR, typename V>
__device__ __forceinline__ void block_fft(V (&v)[NF][E], V* sbuf, const V* __restrict__ tw, int t, int bar = 0) {
  static_assert((P & (P - 1)) == 0 && P >= 2 && P <= kMaxFFT, "P must be a power of two <= 4096");
  static_assert(E >= 2 && E <= 16 && (E & (E - 1)) == 0 && E <= P, "E must be a power of two <= 16");
  static_assert(P / E <= 32 || (P / E) % 32 == 0, "a group barrier spans whole warps");
  // Groups of fewer than 16 threads share a half-warp with their neighbours, whose buffers start on
  // the same bank: the low 4 bits of group g's exchange positions are XORed with (g * 13) & 15
  // (g * 9 for 2-thread groups), which keeps the scatter and gather of neighbouring groups apart
  // (checked for every radix schedule with 2, 4 and 8 threads per group). The XOR permutes each
  // aligned run of 16 positions, so it stays inside a buffer of P >= 16.
  constexpr int T = P / E;
  const int gkey = (bar > 0 && T >= 2 && T < 16 && P >= 16) ? (((bar - 1) * (T == 2 ? 9 : 13)) & 15) : 0;
  fft_passes<P, E, NF, DIR, 1>(v, sbuf, tw, t, bar, gkey);
}

}  // namespace fbst
