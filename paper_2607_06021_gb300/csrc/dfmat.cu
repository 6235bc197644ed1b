// Tall products in double-float arithmetic on the FP32 pipe, for data that are
// exact FP32 values or double-float (hi, lo) pairs of FP32 planes: the
// refinement's recompressions of the residual (stacked FP64 factors split into
// (hi, lo) planes) and of the sum of the trial solution and the correction
// (stacked FP32 factors).  GB300's FP32 pipe is 64x its FP64 pipe.
//
// A product of a = ah + al and b = bh + bl is taken as ah*bh exactly (one FMA
// gives the rounding error) plus the cross terms ah*bl + al*bh (al*bl is below
// 2^-48 relative and dropped); sums are TwoSum-compensated.  The relative error
// of a K-term sum is below ~2 K^2 eps32^2 in the worst case (~1e-13 typically).
//
//  k_gemm_dfx   Out = A * Bm with A FP32 or (hi, lo), Bm FP64 (split into hi, lo
//               when staged), Out FP64, (hi, lo) planes, or the hi plane alone
//               (the product rounded to FP32).
//  k_gram_dd    Gram partials of (hi, lo) data, renormalised after every chunk.
#include <cuda_runtime.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "f64cvt.cuh"
#include "tall.cuh"

namespace lrp {

namespace {
constexpr int DT = 256;        // threads per CTA
constexpr int DK = 16;         // K slice
constexpr int DROWS = 128;     // rows per tile
constexpr int DTILES = 4;      // tiles per CTA
constexpr int DKC = 32;        // Gram rows per chunk
constexpr int DMAX = 64;       // widths served by the Gram kernel

// hi + lo += (ah + al) (bh + bl), see the header.
__device__ __forceinline__ void dd_madd(float ah, float al, float bh, float bl, float& hi, float& lo) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float cr = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, __fadd_rn(pe, cr)));
}

// (hi, lo) <- TwoSum(hi, lo): the same value with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void dd_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(lo, bb));
  hi = s;
}

// (hi, lo) parts of a double: hi = the nearest float, lo = the nearest float to the rest.
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  hi = f64_to_f32_rn(x);
  lo = f64_to_f32_rn(x - f32_to_f64(hi));
}
}  // namespace

// Out(:, c0:c0+32) for the CTA's rows; see the header.  A has mi columns
// (sel_in), Out mo columns (sel_out); 256 threads, each 4 rows x 4 columns.
template <bool OUT_DF>
__global__ void __launch_bounds__(DT) k_gemm_dfx(TallGeom g, const SolveState* __restrict__ st_all,
                                                 Strided<const float> ah, Strided<const float> al, int sel_in,
                                                 Strided<const double> bm, int sel_out, Strided<float> oh,
                                                 Strided<float> ol, Strided<double> o64, int tri) {
  const int slot = blockIdx.z >> 1, side = blockIdx.z & 1;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mi = dim_of(st, side, sel_in), mo = dim_of(st, side, sel_out);
  const int rbase = blockIdx.x * DROWS * DTILES;
  const int c0 = blockIdx.y * 32;
  if (rbase >= g.n || c0 >= mo || mi < 1) return;
  __shared__ __align__(16) float Ash[DK][DROWS];
  __shared__ __align__(16) float Asl[DK][DROWS];
  __shared__ __align__(16) float Bsh[64][32];
  __shared__ __align__(16) float Bsl[64][32];
  const float* Ah = ah.at(slot, side);
  const float* Al = al.base ? al.at(slot, side) : nullptr;
  const double* Bm = bm.at(slot, side);
  // 8 column groups of 4, one per warp, and 32 row groups of 4, one per lane: a
  // warp whose columns lie past the product's width, or (upper-triangular Bm)
  // whose columns all lie before a K slice, skips that work as a whole; it
  // would only add exact zeros.
  constexpr int TX = 8, TY = DT / TX, RI = DROWS / TY;
  static_assert(TX * 32 == DT && TY == 32, "one column group per warp");
  const int tid = threadIdx.x, tx = tid >> 5, ty = tid & 31;
  const bool live = c0 + tx * 4 < mo;
  // an upper-triangular Bm: output column c takes rows k <= c only, so the
  // CTA's 32 columns need k < c0 + 32
  const int klim = tri ? min(mi, c0 + 32) : mi;
  const int nkb = (klim + 63) / 64;
  for (int tile = 0; tile < DTILES; ++tile) {
    const int r0 = rbase + tile * DROWS;
    if (r0 >= g.n) break;
    float hi[RI][4], lo[RI][4];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    for (int kb = 0; kb < klim; kb += 64) {
      const int kend = min(klim, kb + 64);
      if (tile == 0 || nkb > 1) {
        __syncthreads();
        const int kpad = (kend - kb + DK - 1) / DK * DK;
        for (int e = tid; e < kpad * 32; e += DT) {
          const int k = e % kpad, c = e / kpad;
          const int col = c0 + c;
          float h = 0.f, l = 0.f;
          if (kb + k < kend && col < mo) split_double(Bm[(int64_t)col * g.M + kb + k], h, l);
          Bsh[k][c] = h;
          Bsl[k][c] = l;
        }
      }
      for (int k0 = kb; k0 < kend; k0 += DK) {
#pragma unroll
        for (int q = 0; q < (DK * DROWS) / DT; ++q) {
          const int e = tid + DT * q;
          const int kk = e / DROWS, i = e % DROWS;
          const int row = r0 + i, k = k0 + kk;
          const bool ok = row < g.n && k < kend;
          Ash[kk][i] = ok ? Ah[(int64_t)k * g.ld + row] : 0.f;
          Asl[kk][i] = (ok && Al) ? Al[(int64_t)k * g.ld + row] : 0.f;
        }
        __syncthreads();
        if (live && !(tri && c0 + tx * 4 + 3 < k0)) {
#pragma unroll 4
          for (int kk = 0; kk < DK; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&Ash[kk][ty * RI]);
            const float4 l4 = *reinterpret_cast<const float4*>(&Asl[kk][ty * RI]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bsh[k0 - kb + kk][tx * 4]);
            const float4 c4 = *reinterpret_cast<const float4*>(&Bsl[k0 - kb + kk][tx * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, alv[4] = {l4.x, l4.y, l4.z, l4.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w}, blv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) dd_madd(av[i], alv[i], bv[j], blv[j], hi[i][j], lo[i][j]);
          }
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tx * 4 + j;
      if (col >= mo) continue;
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const int row = r0 + ty * RI + i;
        if (row >= g.n) continue;
        const int64_t o = (int64_t)col * g.ld + row;
        if (OUT_DF) {
          const float h = __fadd_rn(hi[i][j], lo[i][j]);
          oh.at(slot, side)[o] = h;
          if (ol.base) ol.at(slot, side)[o] = __fsub_rn(lo[i][j], __fsub_rn(h, hi[i][j]));
        } else {
          o64.at(slot, side)[o] = f32_to_f64(hi[i][j]) + f32_to_f64(lo[i][j]);
        }
      }
    }
  }
}

// Symmetric Gram partials of (hi, lo) data (mx <= 64 columns): 4 x 4 output
// tiles per thread over the row block, row groups summed in shared memory, every
// entry a double-float sum renormalised by TwoSum after every chunk.
__global__ void __launch_bounds__(DT) k_gram_dd(TallGeom g, const SolveState* __restrict__ st_all,
                                                Strided<const float> xh, Strided<const float> xl, int sel,
                                                double* __restrict__ part) {
  constexpr int LDS = DMAX + 4;
  constexpr int TS = 4;
  const int slot = blockIdx.z >> 1, side = blockIdx.z & 1;
  const SolveState& st = st_all[slot];
  if (!st.active) return;
  const int mx = dim_of(st, side, sel);
  if (mx < 1 || mx > DMAX) return;
  const int blk = blockIdx.x;
  const int rbeg = blk * g.rows_per_block;
  const int rend = min(g.n, rbeg + g.rows_per_block);
  const float* Xh = xh.at(slot, side);
  const float* Xl = xl.at(slot, side);
  double* P = part + ((int64_t)(slot * 2 + side) * g.NB + blk) * (int64_t)g.M * g.M;
  constexpr size_t kTile = 2 * DKC * LDS * sizeof(float);
  constexpr size_t kRed = (size_t)DT * TS * TS * sizeof(double);
  __shared__ __align__(16) unsigned char sm[kTile > kRed ? kTile : kRed];
  float (*Sh)[LDS] = reinterpret_cast<float (*)[LDS]>(sm);
  float (*Sl)[LDS] = reinterpret_cast<float (*)[LDS]>(sm + DKC * LDS * sizeof(float));
  const int tx = (mx + TS - 1) / TS;
  const int ntile = tx * (tx + 1) / 2;  // <= 136
  const int G = DT / ntile;
  const int tid = threadIdx.x;
  const int grp = tid / ntile, t0 = tid - grp * ntile;
  const bool own = grp < G;
  int ia = 0, ib = 0;
  if (own) {
    ib = (int)((sqrtf(8.0f * t0 + 1.0f) - 1.0f) * 0.5f);
    while ((ib + 1) * (ib + 2) / 2 <= t0) ++ib;
    while (ib * (ib + 1) / 2 > t0) --ib;
    ia = t0 - ib * (ib + 1) / 2;
  }
  float hi[TS][TS], lo[TS][TS];
#pragma unroll
  for (int i = 0; i < TS; ++i)
#pragma unroll
    for (int j = 0; j < TS; ++j) hi[i][j] = lo[i][j] = 0.f;
  const int wx = tx * TS;
  for (int r = rbeg; r < rend; r += DKC) {
    for (int e = tid; e < DKC * wx; e += DT) {
      const int kk = e % DKC, c = e / DKC;
      const int row = r + kk;
      const bool ok = row < rend && c < mx;
      Sh[kk][c] = ok ? Xh[(int64_t)c * g.ld + row] : 0.f;
      Sl[kk][c] = ok ? Xl[(int64_t)c * g.ld + row] : 0.f;
    }
    __syncthreads();
    if (own) {
      for (int kk = grp; kk < DKC; kk += G) {
        const float4 a4 = *reinterpret_cast<const float4*>(&Sh[kk][TS * ia]);
        const float4 l4 = *reinterpret_cast<const float4*>(&Sl[kk][TS * ia]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Sh[kk][TS * ib]);
        const float4 c4 = *reinterpret_cast<const float4*>(&Sl[kk][TS * ib]);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w}, alv[4] = {l4.x, l4.y, l4.z, l4.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w}, blv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int i = 0; i < TS; ++i)
#pragma unroll
          for (int j = 0; j < TS; ++j) dd_madd(av[i], alv[i], bv[j], blv[j], hi[i][j], lo[i][j]);
      }
#pragma unroll
      for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < TS; ++j) dd_renorm(hi[i][j], lo[i][j]);
    }
    __syncthreads();
  }
  double tot[TS][TS];
#pragma unroll
  for (int i = 0; i < TS; ++i)
#pragma unroll
    for (int j = 0; j < TS; ++j) tot[i][j] = f32_to_f64(hi[i][j]) + f32_to_f64(lo[i][j]);
  double* red = reinterpret_cast<double*>(sm);
  if (own) {
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
      for (int j = 0; j < TS; ++j) red[((size_t)grp * ntile + t0) * TS * TS + i * TS + j] = tot[i][j];
  }
  __syncthreads();
  for (int e = tid; e < ntile * TS * TS; e += DT) {
    const int tt = e / (TS * TS), ij = e % (TS * TS), i = ij / TS, j = ij % TS;
    double v = 0.0;
    for (int q = 0; q < G; ++q) v += red[((size_t)q * ntile + tt) * TS * TS + ij];
    int tb = (int)((sqrtf(8.0f * tt + 1.0f) - 1.0f) * 0.5f);
    while ((tb + 1) * (tb + 2) / 2 <= tt) ++tb;
    while (tb * (tb + 1) / 2 > tt) --tb;
    const int ta = tt - tb * (tb + 1) / 2;
    const int a = TS * ta + i, b = TS * tb + j;
    if (a < mx && b < mx && a <= b) P[(int64_t)b * g.M + a] = v;
  }
}

cudaError_t launch_gemm_dfx(const TallGeom& g, const SolveState* st, Strided<const float> ah, Strided<const float> al,
                            int sel_in, Strided<const double> bm, int sel_out, Strided<float> oh, Strided<float> ol,
                            Strided<double> o64, cudaStream_t s, bool tri) {
  const dim3 grid((g.n + DROWS * DTILES - 1) / (DROWS * DTILES), (g.M + 31) / 32, g.nslots * 2);
  if (o64.base)
    k_gemm_dfx<false><<<grid, DT, 0, s>>>(g, st, ah, al, sel_in, bm, sel_out, oh, ol, o64, tri ? 1 : 0);
  else
    k_gemm_dfx<true><<<grid, DT, 0, s>>>(g, st, ah, al, sel_in, bm, sel_out, oh, ol, o64, tri ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_gram_dd(const TallGeom& g, const SolveState* st, Strided<const float> xh, Strided<const float> xl,
                           int sel, double* part, cudaStream_t s) {
  k_gram_dd<<<dim3(g.NB, 1, g.nslots * 2), DT, 0, s>>>(g, st, xh, xl, sel, part);
  return cudaGetLastError();
}

}  // namespace lrp
