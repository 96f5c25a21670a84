// dsr_programs.cuh -- the built-in region programs: for each, the master's
// sequential code (pushes, fills, parallel calls, pops) and the parallel
// bodies the workers run. W' below is the region width (desc.width, or all
// workers). All integer arithmetic wraps modulo 2^32.
#pragma once

#include "dsr_runtime.cuh"

namespace dsr {

__device__ __forceinline__ const uint32_t *frame_words(uint32_t k) {
  return reinterpret_cast<const uint32_t *>(ctrl()->frames[k].ptr);
}

// ---------------------------------------------------------------------------
// Sec. 6.1, Fig. "Implicitly sharing 8 variables": the frame holds int c[n]
// and the reference to the mapped array a. The master's code block sets
// c_i = 0 and then c_i += i (single thread, as written); the parallel region
// adds the sum of the c_i to a[team*W' + tid].
// ---------------------------------------------------------------------------
struct ProgPaperScalars {
  __device__ static uint32_t ptr_off(uint32_t n) { return (4u * n + 7u) & ~7u; }

  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    const uint32_t n = d.param;
    uint8_t *f = push(d.frame_bytes[0]);
    if (!f) return;
    if (lane_id() == 0) {
      uint32_t *c = reinterpret_cast<uint32_t *>(f);
      for (uint32_t i = 0; i < n; ++i) c[i] = 0;
      for (uint32_t i = 0; i < n; ++i) c[i] += i + 1;
      *reinterpret_cast<uint32_t **>(f + ptr_off(n)) =
          reinterpret_cast<uint32_t *>(e.out + d.out_offset);
    }
    __syncwarp();
    parallel<ProgPaperScalars>(e, 0, region_width(d), 0);
    pop(f);
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t) {
    const uint8_t *f = ctrl()->frames[0].ptr;
    const uint32_t nv = e.d->param;
    uint32_t *a = *reinterpret_cast<uint32_t *const *>(f + ptr_off(nv));
    const uint32_t *c = reinterpret_cast<const uint32_t *>(f);
    uint32_t sum = 0;
    for (uint32_t i = 0; i < nv; ++i) sum += c[i];
    a[e.team * n + tid] += sum;
  }
};

// ---------------------------------------------------------------------------
// Sec. 6.1, Fig. "Implicitly sharing an array": the frame holds k arrays
// int d_m[W']; the master fills them with 10; the parallel region adds
// sum_m d_m[tid] to a[team*W' + tid].
// ---------------------------------------------------------------------------
struct ProgPaperArrays {
  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    uint8_t *f = push(d.frame_bytes[0]);
    if (!f) return;
    uint32_t *w = reinterpret_cast<uint32_t *>(f);
    for (uint32_t i = lane_id(); i < d.frame_bytes[0] / 4u; i += 32u) w[i] = 10u;
    __syncwarp();
    parallel<ProgPaperArrays>(e, 0, region_width(d), 0);
    pop(f);
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t) {
    const uint32_t *dm = frame_words(0);
    uint32_t sum = 0;
    for (uint32_t m = 0; m < e.d->param; ++m) sum += dm[m * n + tid];
    uint32_t *a = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset);
    a[e.team * n + tid] += sum;
  }
};

// ---------------------------------------------------------------------------
// Config 1: R = param sequential regions per team, each pushing int32 s[4]
// from image[r]; out[(r*T + team)*W' + tid] = (s0*tid + s1) ^
// ((s2 >> (tid & 7)) + s3). The master loads region r+1's image before it
// forks region r, so the load overlaps the parallel region.
// ---------------------------------------------------------------------------
struct ProgScalars {
  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    const uint32_t R = d.param, width = region_width(d);
    const uint4 *img = reinterpret_cast<const uint4 *>(e.images + d.image_offset);
    uint4 next = lane_id() == 0 ? __ldg(img) : make_uint4(0, 0, 0, 0);
    for (uint32_t r = 0; r < R; ++r) {
      uint8_t *f = push(16);
      if (!f) return;
      if (lane_id() == 0) {
        *reinterpret_cast<uint4 *>(f) = next;
        if (r + 1 < R) next = __ldg(img + r + 1);
      }
      __syncwarp();
      parallel<ProgScalars>(e, 0, width, r);
      pop(f);
    }
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t r) {
    const uint4 v = *reinterpret_cast<const uint4 *>(ctrl()->frames[0].ptr);
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset);
    o[(static_cast<uint64_t>(r) * e.d->teams + e.team) * n + tid] =
        (v.x * tid + v.y) ^ ((v.z >> (tid & 7u)) + v.w);
  }
};

// ---------------------------------------------------------------------------
// Config 2: D nested master-side calls. Level k pushes F_k = {int32 s[16];
// int32 arr[256]} filled from image[team][k-1] XOR mix32(team*8 + k), with
// F_k.s[0] ^= F_{k-1}.s[15] for k > 1, then forks:
//   k < D: F_k.arr[i] = mix32(F_k.arr[i] + i) for the worker's strided i;
//          after the join the master stores sum(F_k.arr) in F_k.s[15];
//   k = D: out[e] = mix32(e ^ sum_m (F_m.arr[j & 255] ^ F_m.s[j & 15])),
//          e = team*E + j, for the worker's strided j < E (E = param).
// On the way out chk[k-1] = F_k.s[15], then F_k is popped.
// ---------------------------------------------------------------------------
struct ProgNested {
  enum : uint32_t { kUpdate = 0, kInner = 1 };

  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    const uint32_t D = d.depth, width = region_width(d);
    const uint8_t *timg = e.images + d.image_offset + static_cast<uint64_t>(e.team) * D * 1088u;
    for (uint32_t k = 1; k <= D; ++k) {
      bool sm;
      uint8_t *f = push(d.frame_bytes[k - 1], &sm);
      if (!f) return;
      fill(f, sm, timg + (k - 1) * 1088u, 1088u, mix32(e.team * 8u + k));
      if (!team_ok()) return;
      if (k > 1 && lane_id() == 0) reinterpret_cast<uint32_t *>(f)[0] ^= frame_words(k - 2)[15];
      __syncwarp();
      parallel<ProgNested>(e, k < D ? kUpdate : kInner, width, k);
      if (k < D) {
        const uint32_t sum = frame_sum(reinterpret_cast<const uint32_t *>(f) + 16, 256);
        if (lane_id() == 0) reinterpret_cast<uint32_t *>(f)[15] = sum;
        __syncwarp();
      }
    }
    for (uint32_t k = D; k >= 1; --k) {
      const uint8_t *f = ctrl()->frames[k - 1].ptr;
      if (lane_id() == 0) ctrl()->chk[k - 1] = reinterpret_cast<const uint32_t *>(f)[15];
      pop(f);
    }
  }

  __device__ static void body(const Env &e, uint32_t work, uint32_t tid, uint32_t n,
                              uint32_t k) {
    if (work == kUpdate) {
      uint32_t *arr = reinterpret_cast<uint32_t *>(ctrl()->frames[k - 1].ptr) + 16;
      for (uint32_t i = tid; i < 256u; i += n) arr[i] = mix32(arr[i] + i);
      return;
    }
    const uint32_t D = e.d->depth, E = e.d->param;
    const uint32_t *f[DSR_MAX_DEPTH];
#pragma unroll
    for (uint32_t m = 0; m < DSR_MAX_DEPTH; ++m) f[m] = m < D ? frame_words(m) : nullptr;
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset) +
                  static_cast<uint64_t>(e.team) * E;
    const uint32_t ebase = e.team * E;
    for (uint32_t j = tid; j < E; j += n) {
      uint32_t acc = 0;
#pragma unroll
      for (uint32_t m = 0; m < DSR_MAX_DEPTH; ++m)
        if (m < D) acc += f[m][16u + (j & 255u)] ^ f[m][j & 15u];
      o[j] = mix32((ebase + j) ^ acc);
    }
  }
};

// ---------------------------------------------------------------------------
// Config 3: one frame float arr[L] (L = frame_bytes/4) copied from
// image[team]; out[team*W' + tid] = arr[tid] + arr[tid + W'] + ... in index
// order, each addition rounded to fp32 (no contraction).
// ---------------------------------------------------------------------------
struct ProgSweep {
  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    const uint32_t S = d.frame_bytes[0];
    bool sm;
    uint8_t *f = push(S, &sm);
    if (!f) return;
    fill(f, sm, e.images + d.image_offset + static_cast<uint64_t>(e.team) * S, S, 0u);
    if (!team_ok()) return;
    parallel<ProgSweep>(e, 0, region_width(d), 0);
    pop(f);
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t) {
    const float *arr = reinterpret_cast<const float *>(ctrl()->frames[0].ptr);
    const uint32_t L = ctrl()->frames[0].bytes / 4u;
    float acc = 0.0f;
    for (uint32_t i = tid; i < L; i += n) acc = __fadd_rn(acc, arr[i]);
    reinterpret_cast<float *>(e.out + e.d->out_offset)[e.team * n + tid] = acc;
  }
};

// ---------------------------------------------------------------------------
// Config 4/5: D levels of F_k = int32[L_k] filled from the instance's level
// images XOR mix32(salt + team*8 + k), F_k[0] ^= c_{k-1} for k > 1, then:
//   k < D: F_k[w] = mix32(F_k[w] + w) for the worker's strided w; after the
//          join the master sums F_k into c_k (= chk[k-1]);
//   k = D: out[team*W' + tid] = sum over m <= D and the worker's strided w
//          of mix32(F_m[w] ^ (m << 24) ^ w).
// chk[D-1] = F_D[0]; the frames are popped in reverse order.
// ---------------------------------------------------------------------------
struct ProgHetero {
  enum : uint32_t { kUpdate = 0, kInner = 1 };

  __device__ static void master(const Env &e) {
    const dsr_region_desc &d = *e.d;
    const uint32_t D = d.depth, width = region_width(d);
    const uint8_t *img = e.images + d.image_offset;
    uint32_t c_prev = 0;
    for (uint32_t k = 1; k <= D; ++k) {
      const uint32_t S = d.frame_bytes[k - 1];
      bool sm;
      uint8_t *f = push(S, &sm);
      if (!f) return;
      fill(f, sm, img, S, mix32(d.salt + e.team * 8u + k));
      if (!team_ok()) return;
      img += (S + 15u) & ~15u;
      if (k > 1 && lane_id() == 0) reinterpret_cast<uint32_t *>(f)[0] ^= c_prev;
      __syncwarp();
      parallel<ProgHetero>(e, k < D ? kUpdate : kInner, width, k);
      if (k < D) {
        c_prev = frame_sum(reinterpret_cast<const uint32_t *>(f), S / 4u);
        if (lane_id() == 0) ctrl()->chk[k - 1] = c_prev;
      }
    }
    if (lane_id() == 0) ctrl()->chk[D - 1] = frame_words(D - 1)[0];
    for (uint32_t k = D; k >= 1; --k) pop(ctrl()->frames[k - 1].ptr);
  }

  __device__ static void body(const Env &e, uint32_t work, uint32_t tid, uint32_t n,
                              uint32_t k) {
    if (work == kUpdate) {
      uint32_t *f = reinterpret_cast<uint32_t *>(ctrl()->frames[k - 1].ptr);
      const uint32_t L = ctrl()->frames[k - 1].bytes / 4u;
      for (uint32_t w = tid; w < L; w += n) f[w] = mix32(f[w] + w);
      return;
    }
    uint32_t acc = 0;
    for (uint32_t m = 1; m <= k; ++m) {
      const uint32_t *f = frame_words(m - 1);
      const uint32_t L = ctrl()->frames[m - 1].bytes / 4u;
      const uint32_t tag = m << 24;
      for (uint32_t w = tid; w < L; w += n) acc += mix32(f[w] ^ tag ^ w);
    }
    reinterpret_cast<uint32_t *>(e.out + e.d->out_offset)[e.team * n + tid] = acc;
  }
};

}  // namespace dsr
