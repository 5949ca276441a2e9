// bcm_wavelet.cu -- per-cube wavelet compression of a cell field for checkpoints
// (arXiv:1808.04099, section "Data compression": a discrete wavelet transform of every
// cube, one level of quantization, an encoder, one stream with the size of every
// cube's record so that any number of readers can find them).
//
// Transform: log2 B levels of a separable 3-D CDF 5/3 lifting transform of the cube's
// B^3 values (predict d_i = x_{2i+1} - (x_{2i} + x_{2i+2})/2, update
// s_i = x_{2i} + (d_{i-1} + d_i)/4, symmetric at the line ends; passes along x, y, z on
// the low band of each level, coefficients in place, s first then d along each line).
// Quantizer q = rint(c / step).  Encoder (in place of zlib): Golomb-Rice on
// z = zigzag(q) with one parameter k = floor(log2(mean z)) per cube (<= 24); a value
// with u = z >> k below 16 is u one-bits, a zero-bit and the k low bits of z, else 16
// one-bits and the 32 bits of z; bits LSB-first in 32-bit words.  Stream (32-bit
// words): magic "BCMW", version 1, B, n_cubes, 0, 0, step (2 words), the word count of
// every cube record, then the records (a word k | nbits << 5, then ceil(nbits/32)
// payload words).
//
// The codes are integers decided by floating point, so the transform runs in FP64 with
// explicitly rounded operations (no contraction) in one fixed order per line: the same
// arithmetic as a plain sequential implementation, hence the same codes and stream.
// One block per cube: the cube sits in shared memory with rows padded to B + 1 doubles
// (lines along x fall on different banks); a thread per line lifts it; a block scan of
// the code lengths gives every thread's bit offset, and each code is written as one
// <= 48-bit pattern OR-ed into at most three words of a zeroed stream.  Decoding
// stages a record in shared memory and splits its bits among the block's threads (a
// Rice stream has no entry points: the threads find the code boundaries by
// self-synchronisation, see k_wav_decode), then transforms back with the block.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "bcm_internal.cuh"
#include "bcm_kernels.h"

namespace bcm {

namespace {

constexpr uint32_t kMagic = 0x57434d42u;  // "BCMW"
constexpr int kHead = 8;

template <int B>
__device__ __forceinline__ int tix(int i, int j, int k) { return (k * B + j) * (B + 1) + i; }

// element pos of line (a, b) along axis d
template <int B>
__device__ __forceinline__ int line_at(int d, int a, int b, int pos) {
  return d == 0 ? tix<B>(pos, a, b) : (d == 1 ? tix<B>(a, pos, b) : tix<B>(a, b, pos));
}

template <int B>
__device__ void lift_forward(double* X, int d, int a, int b, int m) {
  double tmp[B];
  const int h = m / 2;
  for (int i = 0; i < h; ++i) {
    const double x0 = X[line_at<B>(d, a, b, 2 * i)];
    const double right = (2 * i + 2 < m) ? X[line_at<B>(d, a, b, 2 * i + 2)] : x0;
    const double t = __dmul_rn(0.5, __dadd_rn(x0, right));
    tmp[h + i] = __dsub_rn(X[line_at<B>(d, a, b, 2 * i + 1)], t);
  }
  for (int i = 0; i < h; ++i) {
    const double dl = i > 0 ? tmp[h + i - 1] : tmp[h];
    const double t = __dmul_rn(0.25, __dadd_rn(dl, tmp[h + i]));
    tmp[i] = __dadd_rn(X[line_at<B>(d, a, b, 2 * i)], t);
  }
  for (int i = 0; i < m; ++i) X[line_at<B>(d, a, b, i)] = tmp[i];
}

template <int B>
__device__ void lift_inverse(double* X, int d, int a, int b, int m) {
  double tmp[B];
  const int h = m / 2;
  for (int i = 0; i < h; ++i) {
    const double dl = i > 0 ? X[line_at<B>(d, a, b, h + i - 1)] : X[line_at<B>(d, a, b, h)];
    const double t = __dmul_rn(0.25, __dadd_rn(dl, X[line_at<B>(d, a, b, h + i)]));
    tmp[2 * i] = __dsub_rn(X[line_at<B>(d, a, b, i)], t);
  }
  for (int i = 0; i < h; ++i) {
    const double right = (2 * i + 2 < m) ? tmp[2 * i + 2] : tmp[2 * i];
    const double t = __dmul_rn(0.5, __dadd_rn(tmp[2 * i], right));
    tmp[2 * i + 1] = __dadd_rn(X[line_at<B>(d, a, b, h + i)], t);
  }
  for (int i = 0; i < m; ++i) X[line_at<B>(d, a, b, i)] = tmp[i];
}

__device__ __forceinline__ uint32_t zigzag(int32_t q) {
  return ((uint32_t)q << 1) ^ (uint32_t)(q >> 31);
}
__device__ __forceinline__ int32_t unzigzag(uint32_t z) {
  return (int32_t)(z >> 1) ^ -(int32_t)(z & 1u);
}

__device__ __forceinline__ uint32_t code_len(uint32_t z, int k) {
  const uint32_t u = z >> k;
  return u < 16 ? u + 1 + (uint32_t)k : 48u;
}

// block-wide sum of one 64-bit value per thread; result valid in every thread.  A block
// of fewer than 32 threads (4^3 cubes: 16) shuffles within its own lanes only.
template <int NT>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* red) {
  constexpr unsigned int mask = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
  for (int o = (NT >= 32 ? 16 : NT / 2); o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  unsigned long long s = 0;
  for (int w = 0; w < (NT + 31) / 32; ++w) s += red[w];
  return s;
}

// forward transform, quantization, Rice parameter and record size of one cube
template <int B, class T>
__global__ __launch_bounds__(B * B) void k_wav_forward(const T* __restrict__ f, double step,
                                                       uint32_t* __restrict__ zc,
                                                       uint32_t* __restrict__ cube_nbits,
                                                       uint32_t* __restrict__ cube_k,
                                                       int* __restrict__ err) {
  constexpr int NT = B * B, B3 = B * B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* X = reinterpret_cast<double*>(smem_raw);
  __shared__ unsigned long long red[(NT + 31) / 32];
  const int c = blockIdx.x;
  for (int q = threadIdx.x; q < B3; q += NT)
    X[tix<B>(q % B, (q / B) % B, q / (B * B))] = double(f[(size_t)c * B3 + q]);
  __syncthreads();
  for (int m = B; m >= 2; m /= 2)
    for (int d = 0; d < 3; ++d) {
      if (threadIdx.x < m * m) lift_forward<B>(X, d, threadIdx.x % m, threadIdx.x / m, m);
      __syncthreads();
    }
  unsigned long long zsum = 0;
  for (int q = threadIdx.x; q < B3; q += NT) {
    double r = rint(__ddiv_rn(X[tix<B>(q % B, (q / B) % B, q / (B * B))], step));
    if (!(fabs(r) < 1073741824.0)) {
      atomicOr(err, 1);
      r = 0.0;
    }
    const uint32_t z = zigzag((int32_t)r);
    zc[(size_t)c * B3 + q] = z;
    zsum += z;
  }
  const unsigned long long mean = block_sum_u64<NT>(zsum, red) / (unsigned long long)B3;
  int k = 0;
  while (k < 24 && (mean >> (k + 1)) != 0) ++k;
  unsigned long long bits = 0;
  for (int q = threadIdx.x; q < B3; q += NT) bits += code_len(zc[(size_t)c * B3 + q], k);
  const unsigned long long nbits = block_sum_u64<NT>(bits, red);
  if (threadIdx.x == 0) {
    cube_nbits[c] = (uint32_t)nbits;
    cube_k[c] = (uint32_t)k;
  }
}

// word offsets of the cube records (exclusive scan of their sizes after the head and
// the size table); sizes from cube_nbits (encoding) or from the stream's table
__global__ __launch_bounds__(1024) void k_wav_offsets(const uint32_t* __restrict__ cube_nbits,
                                                      const uint32_t* __restrict__ table,
                                                      int n_cubes, uint32_t* __restrict__ off) {
  __shared__ unsigned long long buf[1024];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = (unsigned long long)kHead + n_cubes;
  __syncthreads();
  for (int base = 0; base < n_cubes; base += 1024) {
    const int c = base + threadIdx.x;
    unsigned long long v = 0;
    if (c < n_cubes) v = cube_nbits ? 1ull + (cube_nbits[c] + 31u) / 32u : table[c];
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const unsigned long long add = threadIdx.x >= o ? buf[threadIdx.x - o] : 0ull;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (c < n_cubes) off[c] = (uint32_t)(carry + buf[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n_cubes] = (uint32_t)carry;
}

// OR a code of at most 48 bits into the payload at bit pos.  Only words that receive a
// set bit are touched: every set bit lies below the record's bit count, so no write
// leaves the record.
__device__ __forceinline__ void put_code(uint32_t* w, unsigned long long pos,
                                         unsigned long long pat) {
  const unsigned int off = (unsigned int)(pos & 31u);
  uint32_t* p = w + (pos >> 5);
  const uint32_t w0 = (uint32_t)(pat << off), w1 = (uint32_t)(pat >> (32 - off));
  const uint32_t w2 = off ? (uint32_t)(pat >> (64 - off)) : 0u;
  if (w0) atomicOr(p, w0);
  if (w1) atomicOr(p + 1, w1);
  if (w2) atomicOr(p + 2, w2);
}

template <int B>
__global__ __launch_bounds__(B * B) void k_wav_encode(const uint32_t* __restrict__ zc,
                                                      const uint32_t* __restrict__ cube_nbits,
                                                      const uint32_t* __restrict__ cube_k,
                                                      const uint32_t* __restrict__ off,
                                                      int n_cubes, double step,
                                                      uint32_t* __restrict__ out) {
  constexpr int NT = B * B, B3 = B * B * B, P = B3 / NT;
  __shared__ unsigned long long scan[NT];
  const int c = blockIdx.x;
  const int k = (int)cube_k[c];
  const uint32_t nbits = cube_nbits[c];
  const size_t rec = off[c];
  if (threadIdx.x == 0) {
    out[kHead + c] = 1u + (nbits + 31u) / 32u;
    out[rec] = (uint32_t)k | (nbits << 5);
    if (c == 0) {
      out[0] = kMagic;
      out[1] = 1u;
      out[2] = (uint32_t)B;
      out[3] = (uint32_t)n_cubes;
      out[4] = out[5] = 0u;
      const unsigned long long sb = (unsigned long long)__double_as_longlong(step);
      out[6] = (uint32_t)sb;
      out[7] = (uint32_t)(sb >> 32);
    }
  }
  // thread t codes values t P .. t P + P - 1: its bit offset is the exclusive scan of
  // the threads' code lengths
  const uint32_t* z = zc + (size_t)c * B3 + (size_t)threadIdx.x * P;
  unsigned long long mine = 0;
  for (int e = 0; e < P; ++e) mine += code_len(z[e], k);
  scan[threadIdx.x] = mine;
  __syncthreads();
  for (int o = 1; o < NT; o <<= 1) {
    const unsigned long long add = threadIdx.x >= o ? scan[threadIdx.x - o] : 0ull;
    __syncthreads();
    scan[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned long long pos = scan[threadIdx.x] - mine;
  uint32_t* w = out + rec + 1;
  for (int e = 0; e < P; ++e) {
    const uint32_t zz = z[e], u = zz >> k;
    unsigned long long pat;
    uint32_t len;
    if (u < 16) {
      const unsigned long long lowk = k ? (zz & ((1u << k) - 1u)) : 0u;
      pat = ((1ull << u) - 1ull) | (lowk << (u + 1));
      len = u + 1 + (uint32_t)k;
    } else {
      pat = 0xFFFFull | ((unsigned long long)zz << 16);
      len = 48;
    }
    put_code(w, pos, pat);
    pos += len;
  }
}

// 64 bits of a staged record from bit p on (W: the record's payload words, then zero
// words)
__device__ __forceinline__ unsigned long long rice_window(const uint32_t* W, uint32_t p) {
  const uint32_t i = p >> 5, sh = p & 31u;
  const unsigned long long lo = (unsigned long long)W[i] | ((unsigned long long)W[i + 1] << 32);
  return sh ? (lo >> sh) | ((unsigned long long)W[i + 2] << (64u - sh)) : lo;
}

// From the code starting at bit p (< lim): past that code, or past the whole run of
// all-zero codes starting there (u = 0 and k zero bits: the value 0; the run is cut
// after its last code that starts before lim, and at tgt when a code of the run starts
// there).  Returns the codes passed; z is the value of a single code (0 for a run).
// Rice with parameter k; 16 leading one-bits mark the escape, whose next 32 bits are z.
__device__ __forceinline__ uint32_t rice_adv(const uint32_t* W, uint32_t& p, uint32_t lim, int k,
                                             uint32_t& z, uint32_t tgt = 0) {
  const unsigned long long win = rice_window(W, p);
  const uint32_t len0 = (uint32_t)k + 1;
  if ((win & ((2ull << k) - 1ull)) == 0) {
    const uint32_t zeros = win ? (uint32_t)(__ffsll((long long)win) - 1) : 64u;
    const uint32_t room = (lim - p + (uint32_t)k) / len0;  // codes starting before lim
    uint32_t m = min(zeros / len0, room);                  // >= 1
    if (tgt > p && (tgt - p) % len0 == 0 && (tgt - p) / len0 <= m) m = (tgt - p) / len0;
    p += m * len0;
    z = 0;
    return m;
  }
  const uint32_t t = (uint32_t)__clzll((long long)__brevll(~win));  // leading one-bits
  if (t < 16) {
    z = (t << k) | (uint32_t)((win >> (t + 1)) & ((1ull << k) - 1ull));
    p += t + len0;
  } else {
    z = (uint32_t)(win >> 16);
    p += 48u;
  }
  return 1;
}

// The new path from ne against the old one from e (which ended at x after n codes)
// through a segment ending at s1, the one behind first; a run of zero codes stops
// where the other path stands only when one of its codes starts there (two paths out
// of step cross a run in one step each).  Where they meet the old path stands; else
// the new one runs to the segment's end.  Returns whether the exit x moved.
__device__ __forceinline__ bool rice_rewalk(const uint32_t* W, int k, uint32_t s1, uint32_t ne,
                                            uint32_t e, uint32_t& x, uint32_t& n) {
  uint32_t pn = ne, po = e, cn = 0, co = 0, z;
  while (true) {
    if (pn >= s1) {  // left the segment without meeting the old path
      const bool moved = pn != x;
      x = pn;
      n = cn;
      return moved;
    }
    if (pn == po) {  // in step: the rest of the old path stands
      n = cn + (n - co);
      return false;
    }
    if (po < pn)
      co += rice_adv(W, po, s1, k, z, pn);
    else
      cn += rice_adv(W, pn, s1, k, z, po);
  }
}

// Entries of a warp's segments: its first lane enters at went, every other lane at the
// exit of the lane before it; a lane whose entry moved re-walks, until no entry moves
// (one lane more is exact per pass).
__device__ __forceinline__ void rice_warp_entries(const uint32_t* W, int k, uint32_t s1,
                                                  uint32_t went, unsigned mask, int lane,
                                                  uint32_t& e, uint32_t& x, uint32_t& n) {
  for (int pass = 0; pass <= 32; ++pass) {
    const uint32_t px = __shfl_up_sync(mask, x, 1);
    const uint32_t ne = lane == 0 ? went : px;
    if (!__any_sync(mask, ne != e)) return;
    if (ne != e) {
      rice_rewalk(W, k, s1, ne, e, x, n);
      e = ne;
    }
  }
}

// decode one record with the block, dequantize, transform back, store the field.
// The record's bits are cut into one segment per thread.  Each thread decodes its
// segment from the segment's first bit as if a code started there; a prefix code falls
// back into step with the true code boundaries after a few codes (the self-
// synchronisation used for parallel Huffman decoding by Klein and Wiseman, 2003).  The
// true entry of a segment is the exit of the one before it: each warp first settles
// the entries of its lanes from its first lane's (shuffles, no block barrier), then
// block rounds hand every warp the exit of the warp before it and the warps whose
// entry moved settle again.  A thread whose entry moved re-walks from it only until the
// new path meets its old one.  Thread 0 starts at bit 0, so after block round r the
// first r + 2 warps are exact.  Runs of all-zero codes, which keep a path out of step
// for as long as they last, are passed in one step each.  An exclusive scan of the
// code counts gives each segment its first index.  Results equal a sequential decode:
// codes past the B^3-th are ignored, and a record whose B^3 codes do not fit in its bit
// count is malformed (error bit 2, its values from the first code that does not fit
// are 0).
template <int B, class T>
__global__ __launch_bounds__(B * B) void k_wav_decode(const uint32_t* __restrict__ in,
                                                      const uint32_t* __restrict__ off,
                                                      size_t words, uint32_t wcap, double step,
                                                      T* __restrict__ f, int* __restrict__ err) {
  constexpr int NT = B * B, B3 = B * B * B, WS = NT < 32 ? NT : 32, NW = NT / WS;
  constexpr unsigned kMask = WS == 32 ? 0xffffffffu : (1u << WS) - 1u;
  constexpr uint32_t kMaxBits = 48u * B3;  // B^3 codes never need more
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* X = reinterpret_cast<double*>(smem_raw);
  uint32_t* W = reinterpret_cast<uint32_t*>(X + B * B * (B + 1));
  __shared__ uint32_t s_wexit[NW], s_cnt[NT];
  __shared__ uint32_t s_head[3];  // bad, k, bit count
  const int c = blockIdx.x, t = threadIdx.x, lane = t % WS, warp = t / WS;
  const size_t rec = off[c];
  if (t == 0) {
    const size_t cw = in[kHead + c];
    bool bad = cw < 1 || rec + cw > words;
    const uint32_t head = bad ? 0u : in[rec];
    const uint32_t nbits = head >> 5;
    const uint32_t nb = nbits < kMaxBits ? nbits : kMaxBits;
    bad = bad || (head & 31u) > 24u || ((size_t)nbits + 31) / 32 + 1 > cw || (nb + 31) / 32 > wcap;
    s_head[0] = bad;
    s_head[1] = head & 31u;
    s_head[2] = nbits;
  }
  // every value 0 until a code says otherwise (the codes of value 0 write nothing)
  for (int q = t; q < B3; q += NT) X[tix<B>(q % B, (q / B) % B, q / (B * B))] = 0.0;
  __syncthreads();
  const int k = (int)s_head[1];
  const uint32_t nbits = s_head[2], nb = nbits < kMaxBits ? nbits : kMaxBits;
  uint32_t valid = 0;
  if (!s_head[0]) {
    const uint32_t nw = (nb + 31) / 32;  // <= the record's payload words and wcap
    for (uint32_t q = t; q < nw + 3; q += NT) W[q] = q < nw ? in[rec + 1 + q] : 0u;
    __syncthreads();
    const uint32_t s0 = (uint32_t)((unsigned long long)nb * t / NT);
    const uint32_t s1 = (uint32_t)((unsigned long long)nb * (t + 1) / NT);
    uint32_t e = s0, x = s0, n = 0, z;
    while (x < s1) n += rice_adv(W, x, s1, k, z);
    // the warp's lanes from its first lane's speculative entry
    rice_warp_entries(W, k, s1, __shfl_sync(kMask, e, 0), kMask, lane, e, x, n);
    if (lane == WS - 1) s_wexit[warp] = x;
    __syncthreads();
    for (int round = 0; round <= NW; ++round) {
      const uint32_t went = warp ? s_wexit[warp - 1] : 0u;
      __syncthreads();
      rice_warp_entries(W, k, s1, went, kMask, lane, e, x, n);
      bool moved = false;
      if (lane == WS - 1 && x != s_wexit[warp]) {
        s_wexit[warp] = x;
        moved = true;
      }
      if (!__syncthreads_or(moved)) break;
    }
    // first index of each segment: exclusive scan of the counts
    s_cnt[t] = n;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
      const uint32_t add = t >= o ? s_cnt[t - o] : 0u;
      __syncthreads();
      s_cnt[t] += add;
      __syncthreads();
    }
    const uint32_t total = s_cnt[NT - 1];
    // the path's last code runs past the bit count when the last exit lies beyond it
    const uint32_t fit = total - (s_wexit[NW - 1] > nbits ? 1u : 0u);
    valid = fit < (uint32_t)B3 ? fit : (uint32_t)B3;
    uint32_t idx = s_cnt[t] - n, p = e;
    while (p < s1) {
      const uint32_t m = rice_adv(W, p, s1, k, z);
      if (z != 0 && idx < valid)  // a single code (m = 1)
        X[tix<B>(idx % B, (idx / B) % B, idx / (B * B))] = __dmul_rn((double)unzigzag(z), step);
      idx += m;
    }
  }
  if (t == 0 && valid < (uint32_t)B3) atomicOr(err, 2);
  __syncthreads();
  for (int m = 2; m <= B; m *= 2)
    for (int d = 2; d >= 0; --d) {
      if (threadIdx.x < m * m) lift_inverse<B>(X, d, threadIdx.x % m, threadIdx.x / m, m);
      __syncthreads();
    }
  for (int q = threadIdx.x; q < B3; q += NT)
    f[(size_t)c * B3 + q] = T(X[tix<B>(q % B, (q / B) % B, q / (B * B))]);
}

template <int B>
constexpr size_t wav_smem() { return sizeof(double) * B * B * (B + 1); }
// the decoder also stages a record: wcap payload words (at most 48 B^3 bits, all B^3
// codes can use) and three zero words
template <int B>
size_t wav_dec_smem(uint32_t wcap) { return wav_smem<B>() + 4 * ((size_t)wcap + 3); }

template <class K>
cudaError_t wav_allow(K kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int B, class T>
cudaError_t compress_t(const Ctx& x, const void* field, double step, uint32_t* zc,
                       uint32_t* cube_nbits, uint32_t* cube_k, uint32_t* off, int* err) {
  auto kf = k_wav_forward<B, T>;
  cudaError_t e = wav_allow(kf, wav_smem<B>());
  if (e != cudaSuccess) return e;
  kf<<<x.g.n_cubes, B * B, wav_smem<B>(), x.stream>>>((const T*)field, step, zc, cube_nbits,
                                                      cube_k, err);
  k_wav_offsets<<<1, 1024, 0, x.stream>>>(cube_nbits, nullptr, x.g.n_cubes, off);
  return cudaGetLastError();
}

template <int B, class T>
cudaError_t decompress_t(const Ctx& x, void* field, const uint32_t* in, size_t words,
                         uint32_t max_payload, double step, uint32_t* off, int* err) {
  k_wav_offsets<<<1, 1024, 0, x.stream>>>(nullptr, in + kHead, x.g.n_cubes, off);
  auto kd = k_wav_decode<B, T>;
  const uint32_t wcap = std::min<uint32_t>(max_payload, 48u * B * B * B / 32u);
  const size_t sm = wav_dec_smem<B>(wcap);
  cudaError_t e = wav_allow(kd, sm);
  if (e != cudaSuccess) return e;
  kd<<<x.g.n_cubes, B * B, sm, x.stream>>>(in, off, words, wcap, step, (T*)field, err);
  return cudaGetLastError();
}

}  // namespace

#define BCM_WAV_DISPATCH(F, ...)                                                          \
  switch (x.B) {                                                                          \
    case 4: return f64 ? F<4, double>(__VA_ARGS__) : F<4, float>(__VA_ARGS__);            \
    case 8: return f64 ? F<8, double>(__VA_ARGS__) : F<8, float>(__VA_ARGS__);            \
    case 16: return f64 ? F<16, double>(__VA_ARGS__) : F<16, float>(__VA_ARGS__);         \
    default: return cudaErrorInvalidValue;                                                \
  }

cudaError_t launch_wavelet_analyze(const Ctx& x, const void* field, int f64, double step,
                                   uint32_t* zc, uint32_t* cube_nbits, uint32_t* cube_k,
                                   uint32_t* off, int* err) {
  BCM_WAV_DISPATCH(compress_t, x, field, step, zc, cube_nbits, cube_k, off, err)
}

cudaError_t launch_wavelet_encode(const Ctx& x, const uint32_t* zc, const uint32_t* cube_nbits,
                                  const uint32_t* cube_k, const uint32_t* off, double step,
                                  uint32_t* out) {
  switch (x.B) {
    case 4:
      k_wav_encode<4><<<x.g.n_cubes, 16, 0, x.stream>>>(zc, cube_nbits, cube_k, off,
                                                        x.g.n_cubes, step, out);
      break;
    case 8:
      k_wav_encode<8><<<x.g.n_cubes, 64, 0, x.stream>>>(zc, cube_nbits, cube_k, off,
                                                        x.g.n_cubes, step, out);
      break;
    case 16:
      k_wav_encode<16><<<x.g.n_cubes, 256, 0, x.stream>>>(zc, cube_nbits, cube_k, off,
                                                          x.g.n_cubes, step, out);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_wavelet_decode(const Ctx& x, void* field, int f64, const uint32_t* in,
                                  size_t words, uint32_t max_payload, double step, uint32_t* off,
                                  int* err) {
  BCM_WAV_DISPATCH(decompress_t, x, field, in, words, max_payload, step, off, err)
}

}  // namespace bcm
