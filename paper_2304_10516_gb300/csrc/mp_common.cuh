// mp_common.cuh -- pieces of the FP16 tensor-core path shared by the
// training/decode kernels (mp_path.cu) and the direct INR ray-marcher
// (render_inr.cu): the shared-memory tile layout, the hash-grid gather into a
// tile, weight staging, the forward MMA chain, fixed-point coordinates and
// the launch layout. Everything has internal linkage: each translation unit
// gets its own copy.
//
// Tile buffers in shared memory hold 128 samples x features as FP16 core
// matrices (8 samples x 8 features, 128 B): feature group g, sample group q
// at byte ((g * 16) + q) * 128. Read along features they are the K-major A
// operand of a layer (M = samples); read along samples they are the MN-major
// operands of the weight-gradient products (K = samples).
#pragma once

#include <algorithm>

#include "dvnr_internal.cuh"
#include "umma.cuh"

namespace dvnr {

namespace {

constexpr int kTile = 128;
#ifndef DVNR_DEC_PAIR
#define DVNR_DEC_PAIR false
#endif
#ifndef DVNR_DEC_GROUP
#define DVNR_DEC_GROUP 2
#endif
#ifndef DVNR_TRAIN_PAIR
#define DVNR_TRAIN_PAIR true
#endif
// CTAs per SM the decode kernel is built for (registers capped to fit)
#ifndef DVNR_DEC_CTAS
#define DVNR_DEC_CTAS 6
#endif
constexpr int kDecodeCtasPerSm = DVNR_DEC_CTAS;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s of SM clock per wait

__device__ __forceinline__ uint32_t tile_off(uint32_t f, uint32_t s) {
  return ((((f >> 3) << 4) + (s >> 3)) << 7) + ((s & 7u) << 4) + ((f & 7u) << 1);
}
// Weight (out o, in i) of a layer with `out` rows: core matrix (o/8, i/8).
__device__ __forceinline__ uint32_t wsm_off(uint32_t o, uint32_t i, uint32_t out) {
  return (((i >> 3) * (out >> 3) + (o >> 3)) << 7) + ((o & 7u) << 4) + ((i & 7u) << 1);
}

struct MpLayout {
  uint32_t smem_wout, smem_w, smem_dz, smem_act, smem_bytes;
  uint32_t dpad;  // encoding width rounded up to 16 (the K of layer 0; features D..dpad-1 are 0)
  uint32_t wbyte[kMaxHidden + 1];   // byte offset of W_k inside the weight area
  uint32_t act_off[kMaxHidden];     // feature offset of H_k in ACT (H_0 = X0)
  uint32_t tmem_cols;
  uint32_t dw_col[kMaxHidden];      // TMEM column of dW_k
  int ctas_per_sm;
  // warp-specialised training kernel (k_mp_train_ws): two X0 tiles (ACT's
  // feature 0 is slot 0's; the hidden activations follow both slots), the
  // targets (2 x 128 floats) and fixed-point coordinates (2 x 128 x 3) of the
  // tiles in the slots, the gather staging of each of its two gathering
  // groups (stage_levels levels each), and the TMEM columns of each slot's
  // dL/d(encoding)
  int32_t ws;
  uint32_t smem_x0[2], smem_tgt, smem_crd, smem_stage;
  int32_t stage_levels;
  uint32_t dx_col[2];
};

// ---------------------------------------------------------------- gathers --
template <int F>
struct HalfVec;
template <>
struct HalfVec<1> {
  static __device__ __forceinline__ void load(const __half* p, float* v) { v[0] = __half2float(__ldg(p)); }
};
template <>
struct HalfVec<2> {
  static __device__ __forceinline__ void load(const __half* p, float* v) {
    const __half2 a = __ldg(reinterpret_cast<const __half2*>(p));
    const float2 f = __half22float2(a);
    v[0] = f.x;
    v[1] = f.y;
  }
};
template <>
struct HalfVec<4> {
  static __device__ __forceinline__ void load(const __half* p, float* v) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <>
struct HalfVec<8> {
  static __device__ __forceinline__ void load(const __half* p, float* v) {
    HalfVec<4>::load(p, v);
    HalfVec<4>::load(p + 4, v + 4);
  }
};

template <int F>
__device__ __forceinline__ void red_add(float* p, const float* g);
template <>
__device__ __forceinline__ void red_add<1>(float* p, const float* g) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(g[0]) : "memory");
}
template <>
__device__ __forceinline__ void red_add<2>(float* p, const float* g) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(g[0]), "f"(g[1]) : "memory");
}
template <>
__device__ __forceinline__ void red_add<4>(float* p, const float* g) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(g[0]), "f"(g[1]),
               "f"(g[2]), "f"(g[3])
               : "memory");
}
template <>
__device__ __forceinline__ void red_add<8>(float* p, const float* g) {
  red_add<4>(p, g);
  red_add<4>(p + 4, g + 4);
}

// Two single-precision products / fused multiply-adds in one instruction
// (mul.rn.f32x2, fma.rn.f32x2 of the sm_100 family); each lane rounds as the
// scalar operation does, so results are bit-identical to the scalar form.
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// Store F halves of one sample row (features f0 .. f0+F-1, same 16-byte row).
template <int F>
__device__ __forceinline__ void st_row(uint8_t* base, uint32_t off, const float* v) {
  if (F == 1) {
    *reinterpret_cast<__half*>(base + off) = __float2half_rn(v[0]);
  } else if (F == 2) {
    *reinterpret_cast<__half2*>(base + off) = __floats2half2_rn(v[0], v[1]);
  } else if (F == 4) {
    uint2 u;
    __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(base + off) = u;
  } else {
    uint4 u;
    __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    __half2 c = __floats2half2_rn(v[4], v[5]), d = __floats2half2_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    u.z = *reinterpret_cast<uint32_t*>(&c);
    u.w = *reinterpret_cast<uint32_t*>(&d);
    *reinterpret_cast<uint4*>(base + off) = u;
  }
}

// Hash-grid encoding of one coordinate, FP16 tables, FP32 interpolation,
// written as FP16 to the sample's row of the ACT tile (feature 0 .. D-1).
// The corner loads of LG levels are issued together so that their latencies
// overlap; with PAIR, x-neighbour corners in an aligned entry pair share one
// load (training samples are scattered, so this saves requests; decoding walks
// the grid in x order, where neighbouring lanes already share lines).
constexpr int kLevelGroup = 4;

// Features D .. dpad-1 of a sample's row (the zero padding of an encoding
// whose width D is not a multiple of 16 up to layer 0's K): F at a time.
template <int F>
__device__ __forceinline__ void zero_pad_rows(int D, int dpad, uint8_t* act, uint32_t s) {
  float z[F];
#pragma unroll
  for (int f = 0; f < F; ++f) z[f] = 0.f;
  for (int f = D; f < dpad; f += F) st_row<F>(act, tile_off((uint32_t)f, s), z);
}

template <int F, bool PAIR = true, int LG = kLevelGroup, bool ZPAD = false>
__device__ __forceinline__ void encode_to_tile(const LevelTab& lv, const __half* __restrict__ tab16,
                                               uint3 m, bool valid, uint8_t* act, uint32_t s,
                                               int dpad = 0) {
  for (int l0 = 0; l0 < lv.L; l0 += LG) {
    float v[LG][8][F];
    float fr[LG][3];
#pragma unroll
    for (int g = 0; g < LG; ++g) {
      const int l = l0 + g;
      const bool on = valid && l < lv.L;
      uint32_t bx = 0, by = 0, bz = 0;
      fr[g][0] = fr[g][1] = fr[g][2] = 0.f;
      if (on) {
        lattice(m.x, lv.N[l], bx, fr[g][0]);
        lattice(m.y, lv.N[l], by, fr[g][1]);
        lattice(m.z, lv.N[l], bz, fr[g][2]);
      }
      if constexpr (PAIR && F <= 2) {
        // corners x and x+1 whose entries form an aligned pair {2j, 2j+1}
        // (every even x on a hashed level, every even index on a dense one)
        // come in one load of both entries
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (on) {
            const uint32_t y = by + (q & 1), z = bz + (q >> 1);
            const uint32_t i0 = corner_index(lv, l, bx, y, z);
            const uint32_t i1 = corner_index(lv, l, bx + 1, y, z);
            const __half* tab = tab16 + lv.off[l];
            if (i1 == (i0 ^ 1u)) {
              float both[2 * F];
              HalfVec<2 * F>::load(tab + (size_t)(i0 & ~1u) * F, both);
              const bool odd = (i0 & 1u) != 0u;  // corner x is the upper entry
#pragma unroll
              for (int f = 0; f < F; ++f) {
                v[g][2 * q][f] = odd ? both[F + f] : both[f];
                v[g][2 * q + 1][f] = odd ? both[f] : both[F + f];
              }
            } else {
              HalfVec<F>::load(tab + (size_t)i0 * F, v[g][2 * q]);
              HalfVec<F>::load(tab + (size_t)i1 * F, v[g][2 * q + 1]);
            }
          } else {
#pragma unroll
            for (int f = 0; f < F; ++f) v[g][2 * q][f] = v[g][2 * q + 1][f] = 0.f;
          }
        }
      } else {
        if (on) {
          uint32_t idx[8];
          corner_indices8(lv, l, bx, by, bz, idx);
          const __half* tab = tab16 + lv.off[l];
#pragma unroll
          for (int k = 0; k < 8; ++k) HalfVec<F>::load(tab + (size_t)idx[k] * F, v[g][k]);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int f = 0; f < F; ++f) v[g][k][f] = 0.f;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < LG; ++g) {
      const int l = l0 + g;
      if (l >= lv.L) break;
      const float fx = fr[g][0], fy = fr[g][1], fz = fr[g][2];
      float acc[F];
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f] = 0.f;
      // w_k = (wx wy) wz, the x-y products formed once for both z
      const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
      if constexpr (F == 2) {
        // the same products and sums, two lanes per instruction
        const float2 xy01 = fmul2(make_float2(gx, fx), make_float2(gy, gy));  // wxy[0], wxy[1]
        const float2 xy23 = fmul2(make_float2(gx, fx), make_float2(fy, fy));  // wxy[2], wxy[3]
        const float2 w2[4] = {fmul2(xy01, make_float2(gz, gz)), fmul2(xy23, make_float2(gz, gz)),
                              fmul2(xy01, make_float2(fz, fz)), fmul2(xy23, make_float2(fz, fz))};
        float2 a2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float w = (k & 1) ? w2[k >> 1].y : w2[k >> 1].x;
          a2 = ffma2(make_float2(w, w), make_float2(v[g][k][0], v[g][k][1]), a2);
        }
        acc[0] = a2.x;
        acc[F - 1] = a2.y;
      } else {
        const float wxy[4] = {gx * gy, fx * gy, gx * fy, fx * fy};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float w = wxy[k & 3] * ((k >> 2) ? fz : gz);
#pragma unroll
          for (int f = 0; f < F; ++f) acc[f] += w * v[g][k][f];
        }
      }
      st_row<F>(act, tile_off((uint32_t)(l * F), s), acc);
    }
  }
  if constexpr (ZPAD) zero_pad_rows<F>(lv.in_dim, dpad, act, s);
}

// Asynchronous copies global -> shared (cp.async, non-bulk): the issuing
// thread does not wait on a register, so a thread can have all of its
// gathers in flight at once. Sizes 4 and 8 need matching alignment of both
// addresses.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bytes of shared staging per level of encode_to_tile_staged (F = 2): four
// x-neighbour corner pairs of 8 bytes for each of the 128 samples.
constexpr uint32_t kStageLevelBytes = 4u * 128u * 8u;

// encode_to_tile for F = 2 with every corner of a round of levels in flight
// at once: the corner pairs (x, x + 1) at the four (y, z) of each level are
// copied asynchronously into shared staging (one 8-byte copy when the two
// entries form an aligned pair, two 4-byte copies otherwise), then after a
// single wait the thread interpolates from its own staged rows. Staging:
// cap_a levels at stage_a, then cap_b at stage_b (regions of the tile
// buffers that are idle during the encode); more levels run in further
// rounds. Only the issuing thread reads its rows, so no barrier is needed.
// One round of encode_to_tile_staged, split so that a tile's copies can be
// issued early and finished later: stage_round issues the corner copies of
// levels l0 .. l1-1, at most 16 (level l0 + r at stage_a + r 4 KB for r < cap_a, else at
// stage_b + (r - cap_a) 4 KB) and returns the bits of the pairs that arrived
// as (x + 1, x); finish_round waits for the copies and writes the levels'
// interpolated features to the thread's ACT row.
__device__ __forceinline__ uint64_t stage_round(const LevelTab& lv, const __half* __restrict__ tab16, uint3 m,
                                                bool valid, uint32_t s, uint8_t* stage_a, int cap_a,
                                                uint8_t* stage_b, int l0, int l1) {
  constexpr int F = 2;
  uint64_t swapped = 0;  // bit 4 (l - l0) + q: the pair arrived as (x + 1, x)
  if (!valid) return 0;
  for (int l = l0; l < l1; ++l) {
    uint32_t bx, by, bz;
    float f_;
    lattice(m.x, lv.N[l], bx, f_);
    lattice(m.y, lv.N[l], by, f_);
    lattice(m.z, lv.N[l], bz, f_);
    const int r = l - l0;
    const uint32_t lvl = umma::smem_u32(r < cap_a ? stage_a + (uint32_t)r * kStageLevelBytes
                                                  : stage_b + (uint32_t)(r - cap_a) * kStageLevelBytes);
    const __half* tab = tab16 + lv.off[l];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t y = by + (q & 1), z = bz + (q >> 1);
      const uint32_t i0 = corner_index(lv, l, bx, y, z);
      const uint32_t i1 = corner_index(lv, l, bx + 1, y, z);
      const uint32_t dst = lvl + ((uint32_t)q * 128u + s) * 8u;
      if (i1 == (i0 ^ 1u)) {
        cp_async8(dst, tab + (size_t)(i0 & ~1u) * F);
        if (i0 & 1u) swapped |= 1ull << (4 * r + q);
      } else {
        cp_async4(dst, tab + (size_t)i0 * F);
        cp_async4(dst + 4u, tab + (size_t)i1 * F);
      }
    }
  }
  return swapped;
}

__device__ __forceinline__ void finish_round(const LevelTab& lv, uint3 m, bool valid, uint8_t* act, uint32_t s,
                                             const uint8_t* stage_a, int cap_a, const uint8_t* stage_b, int l0,
                                             int l1, uint64_t swapped) {
  constexpr int F = 2;
  cp_async_wait_all();
  for (int l = l0; l < l1; ++l) {
    float acc[F] = {0.f, 0.f};
    if (valid) {
      uint32_t b_;
      float fx, fy, fz;
      lattice(m.x, lv.N[l], b_, fx);
      lattice(m.y, lv.N[l], b_, fy);
      lattice(m.z, lv.N[l], b_, fz);
      const int r = l - l0;
      const uint8_t* lvl = r < cap_a ? stage_a + (uint32_t)r * kStageLevelBytes
                                     : stage_b + (uint32_t)(r - cap_a) * kStageLevelBytes;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint2 raw = *reinterpret_cast<const uint2*>(lvl + ((uint32_t)q * 128u + s) * 8u);
        const bool sw = (swapped >> (4 * r + q)) & 1ull;
        const uint32_t c0 = sw ? raw.y : raw.x, c1 = sw ? raw.x : raw.y;  // corners x, x + 1
        const float2 v0 = __half22float2(*reinterpret_cast<const __half2*>(&c0));
        const float2 v1 = __half22float2(*reinterpret_cast<const __half2*>(&c1));
        // the weights and the order of the sums of encode_to_tile, so both
        // give the same encoding bit for bit
        const float wy = (q & 1) ? fy : 1.f - fy, wz = (q >> 1) ? fz : 1.f - fz;
        const float w0 = ((1.f - fx) * wy) * wz, w1 = (fx * wy) * wz;
        acc[0] += w0 * v0.x;
        acc[1] += w0 * v0.y;
        acc[0] += w1 * v1.x;
        acc[1] += w1 * v1.y;
      }
    }
    st_row<F>(act, tile_off((uint32_t)(l * F), s), acc);
  }
}

__device__ __forceinline__ void encode_to_tile_staged(const LevelTab& lv, const __half* __restrict__ tab16,
                                                      uint3 m, bool valid, uint8_t* act, uint32_t s,
                                                      uint8_t* stage_a, int cap_a, uint8_t* stage_b,
                                                      int cap_b) {
  // at most 16 levels per round: the swap bits of a round fit 64 bits
  const int cap = min(cap_a + cap_b, 16);
  for (int l0 = 0; l0 < lv.L; l0 += cap) {
    const int l1 = min(lv.L, l0 + cap);
    const uint64_t swapped = stage_round(lv, tab16, m, valid, s, stage_a, cap_a, stage_b, l0, l1);
    finish_round(lv, m, valid, act, s, stage_a, cap_a, stage_b, l0, l1, swapped);
  }
}

// One 16-column chunk of dL/d(encoding) (levels c/F .. c/F + 16/F - 1); with
// GUARD, levels at or past L (the zero padding of the last chunk) are skipped.
template <int F, bool GUARD>
__device__ __forceinline__ bool scatter_chunk(const LevelTab& lv, float* __restrict__ grad, uint3 m,
                                              const float (&d)[16], int c) {
  bool bad = false;
  constexpr int LPC = 16 / F;  // levels per 16-column chunk
#pragma unroll
  for (int q = 0; q < LPC; ++q) {
    const int l = c / F + q;
    if (GUARD && l >= lv.L) break;
    uint32_t bx, by, bz;
    float fx, fy, fz;
    lattice(m.x, lv.N[l], bx, fx);
    lattice(m.y, lv.N[l], by, fy);
    lattice(m.z, lv.N[l], bz, fz);
    float* tab = grad + lv.off[l];
#pragma unroll
    for (int f = 0; f < F; ++f) bad |= !isfinite(d[q * F + f]);
    if constexpr (F <= 2) {
      // x-neighbour corners whose entries form an aligned pair {2j, 2j+1}
      // go out as one vector reduction of both entries
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t y = by + (r & 1), z = bz + (r >> 1);
        const float wyz = ((r & 1) ? fy : 1.f - fy) * ((r >> 1) ? fz : 1.f - fz);
        const float w0 = (1.f - fx) * wyz, w1 = fx * wyz;
        const uint32_t i0 = corner_index(lv, l, bx, y, z);
        const uint32_t i1 = corner_index(lv, l, bx + 1, y, z);
        if (i1 == (i0 ^ 1u)) {
          float g[2 * F];
          const bool odd = (i0 & 1u) != 0u;
#pragma unroll
          for (int f = 0; f < F; ++f) {
            g[f] = (odd ? w1 : w0) * d[q * F + f];
            g[F + f] = (odd ? w0 : w1) * d[q * F + f];
          }
          red_add<2 * F>(tab + (size_t)(i0 & ~1u) * F, g);
        } else {
          float g0[F], g1[F];
#pragma unroll
          for (int f = 0; f < F; ++f) {
            g0[f] = w0 * d[q * F + f];
            g1[f] = w1 * d[q * F + f];
          }
          red_add<F>(tab + (size_t)i0 * F, g0);
          red_add<F>(tab + (size_t)i1 * F, g1);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float w = ((k & 1) ? fx : 1.f - fx) * (((k >> 1) & 1) ? fy : 1.f - fy) *
                        (((k >> 2) & 1) ? fz : 1.f - fz);
        const uint32_t idx =
            corner_index(lv, l, bx + (k & 1), by + ((k >> 1) & 1), bz + ((k >> 2) & 1));
        float g[F];
#pragma unroll
        for (int f = 0; f < F; ++f) g[f] = w * d[q * F + f];
        red_add<F>(tab + (size_t)idx * F, g);
      }
    }
  }
  return bad;
}

// Backward of the encoding: dL/d(encoding) is read from TMEM (16 columns
// at a time, the warp-collective load runs on every lane) and each level's
// gradient times the trilinear weights is added to its 8 corner entries
// with vector reductions. Returns true if a non-finite value was seen.
// Load one model's FP16 weights into the core-matrix weight area and w_out
// (as FP32) into s_wout.
// W_0 takes lay.dpad input columns, those past D zero.
// Weights of one model into shared memory, by threads t0 .. t0 + nt - 1 of
// the block (all of them by default).
__device__ void load_weights(const __half* __restrict__ theta16, const int64_t* w_off, int D, int H,
                             int W, const MpLayout& lay, uint8_t* smem, int t0 = -1, int nt = 0) {
  if (t0 < 0) {
    t0 = (int)threadIdx.x;
    nt = (int)blockDim.x;
  }
  uint8_t* s_w = smem + lay.smem_w;
  float* s_wout = reinterpret_cast<float*>(smem + lay.smem_wout);
  for (int k = 0; k < H; ++k) {
    const int in = k == 0 ? D : W;
    const __half* src = theta16 + w_off[k];
    uint8_t* dst = s_w + lay.wbyte[k];
    for (int e = t0; e < W * in; e += nt) {
      const int o = e / in, i = e - o * in;
      *reinterpret_cast<__half*>(dst + wsm_off(o, i, W)) = src[e];
    }
    if (k == 0) {
      for (int e = t0; e < W * ((int)lay.dpad - D); e += nt) {
        const int w = (int)lay.dpad - D, o = e / w, i = D + (e - o * w);
        *reinterpret_cast<__half*>(dst + wsm_off(o, i, W)) = __float2half(0.f);
      }
    }
  }
  for (int j = t0; j < W; j += nt) s_wout[j] = __half2float(theta16[w_off[H] + j]);
}

// Forward MMA chain of layer k: scratch[0:W) = A x W_k^T, A the tile at
// shared address a0 (in features).
__device__ __forceinline__ void issue_forward_at(uint32_t tmem, uint32_t a0, const uint8_t* smem,
                                                 const MpLayout& lay, int k, int in, int W) {
  const uint32_t b0 = umma::smem_u32(smem + lay.smem_w + lay.wbyte[k]);
  const uint32_t id = umma::idesc_f16(kTile, W, 0, 0);
  const uint32_t wb = (uint32_t)(W >> 3) * 128u;
  for (int kk = 0; kk < in / 16; ++kk) {
    const uint64_t a = umma::sdesc(a0 + kk * 4096u, 2048u, 128u);
    const uint64_t b = umma::sdesc(b0 + kk * 2u * wb, wb, 128u);
    umma::mma_f16(tmem, a, b, id, kk > 0);
  }
}
// ... with A = ACT(k).
__device__ __forceinline__ void issue_forward(uint32_t tmem, const uint8_t* smem, const MpLayout& lay,
                                              int k, int in, int W) {
  issue_forward_at(tmem, umma::smem_u32(smem + lay.smem_act) + (lay.act_off[k] >> 3) * 2048u, smem, lay, k,
                   in, W);
}


// Unit-domain fixed-point coordinates of decoding: a global voxel position g
// of a model whose stored block starts at `origin` with n voxels, and the
// stored voxel j itself.
__device__ __forceinline__ uint32_t dec_unit_to_fixed(float g, float origin, int64_t n) {
  if (n < 2) return 0u;
  float u = (g - origin) / (float)(n - 1);
  u = fminf(fmaxf(u, 0.f), 1.f);
  return (uint32_t)__float2uint_rn(u * 16777216.0f);
}
// round(j / (n - 1) * 2^24) = floor((2^25 j + n - 1) / (2 (n - 1))); fd divides
// by 2 (n - 1)
__device__ __forceinline__ uint32_t dec_grid_fixed(uint64_t j, int64_t n, const FastDiv& fd) {
  if (n < 2) return 0u;
  return (uint32_t)fdiv(2 * j * (uint64_t)kFixOne + (uint64_t)(n - 1), fd);
}


int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Layout of k_mp_train_ws (F = 2, encodings of at most 64 features, one
// CTA per SM): false when the configuration exceeds 227 KB of shared memory
// or 512 TMEM columns.
bool make_layout_ws(const dvnr_model m, MpLayout& lay);

uint32_t pow2_cols(uint32_t c) {
  uint32_t p2 = 32;
  while (p2 < c) p2 <<= 1;
  return p2;
}

bool make_layout(const dvnr_model m, bool train, MpLayout& lay) {
  const int W = m->mlp.width, H = m->mlp.n_hidden;
  const int D = (m->lv.in_dim + 15) / 16 * 16;  // layer 0's K: the encoding padded with zeros
  lay = MpLayout{};
  lay.dpad = (uint32_t)D;
  uint32_t off = 64;  // mbarrier, TMEM slot, abort flag, spare
  lay.smem_wout = off;
  off += 64 * 4;
  off = (off + 127) / 128 * 128;
  lay.smem_w = off;
  uint32_t wb = 0;
  for (int k = 0; k < H; ++k) {
    lay.wbyte[k] = wb;
    wb += (uint32_t)W * (k == 0 ? D : W) * 2;
  }
  off += wb;
  off = (off + 1023) / 1024 * 1024;
  const uint32_t feat_bytes = 2048 / 8;  // one feature across 128 samples, per 8-feature group
  if (train) {
    lay.smem_dz = off;
    off += (uint32_t)H * W * feat_bytes;
  }
  lay.smem_act = off;
  lay.act_off[0] = 0;
  if (!train) {
    // inference keeps one activation tile: the epilogue of layer k writes
    // H_(k+1) over the layer's input once its product has completed (the
    // commit's mbarrier covers the operand reads), so that more CTAs fit on
    // an SM
    for (int k = 1; k < H; ++k) lay.act_off[k] = 0u;
    off += (uint32_t)std::max(D, W) * feat_bytes;
  } else {
    for (int k = 1; k < H; ++k) lay.act_off[k] = (uint32_t)D + (uint32_t)(k - 1) * W;
    off += ((uint32_t)D + (uint32_t)(H - 1) * W) * feat_bytes;
  }
  if (train) {
    // the weight-gradient product of dZ_H reads 128 features from its start
    const uint32_t need = lay.smem_dz + ((uint32_t)(H - 1) * W + 128) * feat_bytes;
    off = std::max(off, need);
  }
  lay.smem_bytes = (off + 1023) / 1024 * 1024;
  const uint32_t scratch = (uint32_t)std::max(W, D);
  uint32_t col = scratch;
  if (train) {
    for (int k = 0; k < H; ++k) {
      lay.dw_col[k] = col;
      col += (uint32_t)(k == 0 ? D : W);
    }
  }
  lay.tmem_cols = pow2_cols(col);
  if (lay.tmem_cols > 512 || lay.smem_bytes > 227 * 1024) return false;
  const int by_smem = (int)((228 * 1024) / (lay.smem_bytes + 1024));
  const int by_tmem = (int)(512 / lay.tmem_cols);
  lay.ctas_per_sm = std::max(1, std::min(std::min(by_smem, by_tmem), train ? 2 : kDecodeCtasPerSm));
  return true;
}

bool make_layout_ws(const dvnr_model m, MpLayout& lay) {
  const int W = m->mlp.width, H = m->mlp.n_hidden;
  const int D = (m->lv.in_dim + 15) / 16 * 16;
  lay = MpLayout{};
  if (m->lv.F != 2 || D > 64) return false;
  lay.ws = 1;
  lay.dpad = (uint32_t)D;
  // mbarriers (tensor core, slot full x2, dL/dX0 ready x2, dL/dX0 read x2,
  // teardown), TMEM slot, abort flag, the gathering threads' current model
  uint32_t off = 128;
  lay.smem_wout = off;
  off += 64 * 4;
  off = (off + 127) / 128 * 128;
  lay.smem_w = off;
  uint32_t wb = 0;
  for (int k = 0; k < H; ++k) {
    lay.wbyte[k] = wb;
    wb += (uint32_t)W * (k == 0 ? D : W) * 2;
  }
  off += wb;
  off = (off + 1023) / 1024 * 1024;
  const uint32_t feat_bytes = 2048 / 8;
  lay.smem_act = off;
  lay.smem_x0[0] = off;
  lay.smem_x0[1] = off + (uint32_t)D * feat_bytes;
  lay.act_off[0] = 0;
  for (int k = 1; k < H; ++k) lay.act_off[k] = 2u * (uint32_t)D + (uint32_t)(k - 1) * W;
  off += (2u * (uint32_t)D + (uint32_t)(H - 1) * W) * feat_bytes;
  // dZ last: the weight-gradient product of dZ_H reads 128 features from its
  // start (rows past W land in TMEM lanes that are never read), and the rows
  // past the dZ tiles are padding here, not X0 slots that the gathering
  // groups may be writing meanwhile
  lay.smem_dz = off;
  off += (uint32_t)H * W * feat_bytes;
  off = std::max(off, lay.smem_dz + ((uint32_t)(H - 1) * W + 128) * feat_bytes);
  lay.smem_tgt = off;
  off += 2 * 128 * 4;
  lay.smem_crd = off;
  off += 2 * 128 * 12;
  off = (off + 1023) / 1024 * 1024;
  // the two gathering groups' staging areas, as many levels per round as fit
  lay.smem_stage = off;
  const int fit = (int)(((227u * 1024u > off) ? 227u * 1024u - off : 0u) / (2u * kStageLevelBytes));
  lay.stage_levels = std::min(std::min(m->lv.L, 16), fit);
  if (lay.stage_levels < 1) return false;
  off += 2u * (uint32_t)lay.stage_levels * kStageLevelBytes;
  lay.smem_bytes = (off + 1023) / 1024 * 1024;
  uint32_t col = (uint32_t)std::max(W, D);
  for (int k = 0; k < H; ++k) {
    lay.dw_col[k] = col;
    col += (uint32_t)(k == 0 ? D : W);
  }
  lay.dx_col[0] = col;
  col += (uint32_t)D;
  lay.dx_col[1] = col;
  col += (uint32_t)D;
  lay.tmem_cols = pow2_cols(col);
  lay.ctas_per_sm = 1;
  return lay.tmem_cols <= 512 && lay.smem_bytes <= 227 * 1024;
}

// CTAs of `kernel` resident per SM at `threads` threads and `smem` bytes of
// dynamic shared memory, from the kernel's registers and shared memory
// against the SM's register file and shared memory (1 KB reserved per CTA),
// capped by `cap`: the grid of a persistent launch is this times the SM
// count, one full wave. (The runtime's occupancy query answers 1 for these
// kernels although 6 run side by side, so the limits are applied here.)
template <class K>
int resident_ctas(K kernel, int threads, size_t smem, int cap) {
  cudaFuncAttributes fa{};
  int dev = 0, regs_sm = 65536, smem_sm = 228 * 1024;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * threads;
  const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : cap;
  const int by_smem = (int)((size_t)smem_sm / (smem + fa.sharedSizeBytes + 1024));
  return std::max(1, std::min(std::min(by_regs, by_smem), cap));
}

}  // namespace

}  // namespace dvnr

#define DVNR_WF_DISPATCH(W, F, FN, ...)                         \
  do {                                                          \
    const int w_ = (W), f_ = (F);                               \
    if (w_ == 16 && f_ == 1) FN<16, 1>(__VA_ARGS__);            \
    else if (w_ == 16 && f_ == 2) FN<16, 2>(__VA_ARGS__);       \
    else if (w_ == 16 && f_ == 4) FN<16, 4>(__VA_ARGS__);       \
    else if (w_ == 16 && f_ == 8) FN<16, 8>(__VA_ARGS__);       \
    else if (w_ == 32 && f_ == 1) FN<32, 1>(__VA_ARGS__);       \
    else if (w_ == 32 && f_ == 2) FN<32, 2>(__VA_ARGS__);       \
    else if (w_ == 32 && f_ == 4) FN<32, 4>(__VA_ARGS__);       \
    else if (w_ == 32 && f_ == 8) FN<32, 8>(__VA_ARGS__);       \
    else if (w_ == 64 && f_ == 1) FN<64, 1>(__VA_ARGS__);       \
    else if (w_ == 64 && f_ == 2) FN<64, 2>(__VA_ARGS__);       \
    else if (w_ == 64 && f_ == 4) FN<64, 4>(__VA_ARGS__);       \
    else if (w_ == 64 && f_ == 8) FN<64, 8>(__VA_ARGS__);       \
  } while (0)
