// Row kernels: embed, crop and product over tensors of different shapes.
//
// The paper's TRIOT unrolls the loop nest at compile time for every dimension up to a
// maximum and picks the instantiation at run time (Algorithms 5-8).  Here the nest of the
// OUTER axes becomes a grid of tiles: each CTA takes a tile of consecutive rows (or one
// segment of a long row), decodes every row of the tile once -- the flat-to-tuple step of
// Algorithm 4, with magic-multiplier division -- into per-row offsets in shared memory
// (the Horner/stride sum of Section 1 for each tensor), and then streams the contiguous
// innermost axis with 128-bit accesses.  The number of outer axes is a template
// parameter (one instantiation per rank, chosen by the host's dispatch table, Alg 7).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace triot {

template <typename T>
struct alignas(16) Vec16 {
  T v[16 / sizeof(T)];
};

template <typename T>
__device__ __forceinline__ Vec16<T> ld16(const T* p) {
  return *reinterpret_cast<const Vec16<T>*>(p);
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const Vec16<T>& v) {
  *reinterpret_cast<Vec16<T>*>(p) = v;
}

// ------------------------------------------------------------------ products
// f64 / f32: one IEEE multiply, round to nearest even.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// f16: the product of two halves has at most 22 significant bits and magnitude in
// [2^-48, 2^32], so the f32 product is exact and one rounding to f16 is the correctly
// rounded product.
__device__ __forceinline__ __half mul_rn(__half a, __half b) {
  return __float2half_rn(__fmul_rn(__half2float(a), __half2float(b)));
}

// bf16: the f32 product is exact while its magnitude is at least 2^-126.  Below that the
// f32 product may already be rounded, so the product is formed scaled by 2^128 (exact
// for every magnitude that can round to a non-zero bf16) and rounded on bf16's
// subnormal grid (spacing 2^-133 there, 2^-5 after scaling) with rintf, which rounds to
// nearest even.  On that grid the bf16 encoding of k * 2^-133 is k itself for k <= 256.
__device__ __forceinline__ __nv_bfloat16 mul_rn(__nv_bfloat16 a, __nv_bfloat16 b) {
  const float fa = __bfloat162float(a), fb = __bfloat162float(b);
  const float f = __fmul_rn(fa, fb);
  if (fabsf(f) < 0x1p-125f) {
    const float fs = __fmul_rn(__fmul_rn(fa, 0x1p64f), __fmul_rn(fb, 0x1p64f));
    const unsigned k = (unsigned)rintf(fabsf(fs) * 32.0f);
    const unsigned short sign =
        (unsigned short)((__bfloat16_as_ushort(a) ^ __bfloat16_as_ushort(b)) & 0x8000u);
    return __ushort_as_bfloat16((unsigned short)(sign | k));
  }
  return __float2bfloat16_rn(f);
}

// ------------------------------------------------------------------ row decode
// Flat row index -> offsets of the row in A and B (and, for embed, whether the row's
// tuple lies inside x).  Digits are peeled innermost first as in Algorithm 4; each digit
// multiplies the tensor's stride for that axis.
template <int OP, int NOUT, bool AS>
__device__ __forceinline__ RowInfo decode_row_impl(const RowGeom& g, long long r) {
  // AS: A's row offset from its strides (the product, or a view of a larger tensor);
  // otherwise A is dense and its row offset is r * inner
  long long oa = 0, ob = 0;
  bool inside = true;
  if (g.rows32) {
    uint32_t rem = (uint32_t)r;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      uint32_t t;
      if (k + 1 < NOUT) {
        const uint32_t q = fdiv(rem, g.div[k]);
        t = rem - q * g.div[k].d;
        rem = q;
      } else {
        t = rem;
      }
      if (AS) oa += (long long)t * g.sa[k];
      ob += (long long)t * g.sb[k];
      if ((OP == ROW_EMBED || OP == ROW_EMBED_S)) inside = inside && ((long long)t < g.bound[k]);
    }
  } else {
    long long rem = r;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      long long t;
      if (k + 1 < NOUT) {
        const long long q = rem / g.ext[k];
        t = rem - q * g.ext[k];
        rem = q;
      } else {
        t = rem;
      }
      if (AS) oa += t * g.sa[k];
      ob += t * g.sb[k];
      if ((OP == ROW_EMBED || OP == ROW_EMBED_S)) inside = inside && (t < g.bound[k]);
    }
  }
  RowInfo ri;
  ri.a = AS ? oa : r * g.inner;
  ri.b = ((OP == ROW_EMBED || OP == ROW_EMBED_S) && !inside) ? -1 : ob;
  return ri;
}

template <int OP, int NOUT>
__device__ __forceinline__ RowInfo decode_row(const RowGeom& g, long long r) {
  return decode_row_impl<OP, NOUT, OP == ROW_PRODUCT || OP == ROW_EMBED_S>(g, r);
}

// ------------------------------------------------------------------ the kernel
//
// Grid-stride loop over tiles.  Dynamic shared memory holds one RowInfo per row of a tile.
template <int OP, typename T, int NOUT>
__global__ void __launch_bounds__(1024) rows_kernel(const __grid_constant__ RowGeom g,
                                                    T* __restrict__ A,
                                                    const T* __restrict__ B) {
  extern __shared__ RowInfo rinfo[];
  constexpr int VEC = 16 / int(sizeof(T));
  constexpr int U = 4;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    long long row0, nrows, col0, E;
    if (g.segs_per_row == 1) {
      row0 = tile * g.rows_per_tile;
      nrows = g.rows - row0 < g.rows_per_tile ? g.rows - row0 : g.rows_per_tile;
      col0 = 0;
      E = nrows * g.inner;
    } else {
      row0 = tile / g.segs_per_row;
      col0 = (tile - row0 * g.segs_per_row) * g.seg_len;
      nrows = 1;
      E = g.inner - col0 < g.seg_len ? g.inner - col0 : g.seg_len;
    }
    for (long long q = tid; q < nrows; q += nth) rinfo[q] = decode_row<OP, NOUT>(g, row0 + q);
    __syncthreads();

    if (g.path != PATH_GEN) {
      // Every slot of VEC elements lies inside one row; E and the row starts are multiples
      // of VEC, and A (and for PATH_VEC also B) rows start 16-byte aligned.
      const int nslots = int(E / VEC);
      for (int s0 = tid; s0 < nslots; s0 += nth * U) {
        RowInfo ri[U];
        long long c[U];
        Vec16<T> va[U], vb[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int s = s0 + u * nth;
          ok[u] = s < nslots;
          const long long e = (long long)(ok[u] ? s : 0) * VEC;
          long long q;
          if (g.segs_per_row == 1) {
            uint32_t cc;
            q = fdivmod((uint32_t)e, g.inner_div, cc);
            c[u] = cc;
          } else {
            q = 0;
            c[u] = col0 + e;
          }
          ri[u] = rinfo[q];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
          if constexpr (OP == ROW_PRODUCT) va[u] = ld16(A + ri[u].a + c[u]);
          if constexpr ((OP == ROW_EMBED || OP == ROW_EMBED_S)) {
            if (ri[u].b >= 0 && c[u] < g.b_inner) {
              if (g.path == PATH_VEC) {
                vb[u] = ld16(B + ri[u].b + c[u]);
              } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                  vb[u].v[j] = (c[u] + j < g.b_inner) ? B[ri[u].b + c[u] + j] : T(0);
              }
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j) vb[u].v[j] = T(0);
            }
          } else {
            if (g.path == PATH_VEC) {
              vb[u] = ld16(B + ri[u].b + c[u]);
            } else {
#pragma unroll
              for (int j = 0; j < VEC; ++j) vb[u].v[j] = B[ri[u].b + c[u] + j];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
          T* dst = A + ri[u].a + c[u];
          if constexpr (OP == ROW_PRODUCT) {
            Vec16<T> o;
#pragma unroll
            for (int j = 0; j < VEC; ++j) o.v[j] = mul_rn(va[u].v[j], vb[u].v[j]);
            st16(dst, o);
          } else if ((OP == ROW_EMBED || OP == ROW_EMBED_S) && g.nopad) {
            if (ri[u].b >= 0 && c[u] < g.b_inner) {
              if (c[u] + VEC <= g.b_inner) {
                st16(dst, vb[u]);
              } else {
#pragma unroll
                for (int j = 0; j < VEC; ++j)
                  if (c[u] + j < g.b_inner) dst[j] = vb[u].v[j];
              }
            }
          } else {
            st16(dst, vb[u]);
          }
        }
      }
    } else {
      // Generic path: one element per slot (rows of any length, any alignment); the U
      // slots' loads are all issued before any store, so they are in flight together.
      for (long long e0 = tid; e0 < E; e0 += (long long)nth * U) {
        long long ia[U], ib[U];
        bool ok[U], in[U];
        T va[U], vb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const long long e = e0 + (long long)u * nth;
          ok[u] = e < E;
          long long q = 0, c;
          if (g.segs_per_row == 1) {
            uint32_t cc;
            q = fdivmod((uint32_t)(ok[u] ? e : 0), g.inner_div, cc);
            c = cc;
          } else {
            c = col0 + (ok[u] ? e : 0);
          }
          const RowInfo ri = rinfo[q];
          ia[u] = ri.a + c;
          ib[u] = ri.b + c;
          in[u] = (OP == ROW_EMBED || OP == ROW_EMBED_S) ? (ri.b >= 0 && c < g.b_inner) : true;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          vb[u] = T(0);
          if (ok[u] && in[u]) vb[u] = B[ib[u]];
          if constexpr (OP == ROW_PRODUCT) {
            if (ok[u]) va[u] = A[ia[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
          if constexpr (OP == ROW_PRODUCT) {
            A[ia[u]] = mul_rn(va[u], vb[u]);
          } else if constexpr (OP == ROW_EMBED || OP == ROW_EMBED_S) {
            if (in[u] || !g.nopad) A[ia[u]] = vb[u];  // vb is +0 outside x
          } else {
            A[ia[u]] = vb[u];
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace triot
