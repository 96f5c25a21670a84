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
  static constexpr uint32_t kProgram = DSR_PROG_PAPER_SCALARS;
  static constexpr bool kDense = false;
  __device__ static uint32_t ptr_off(uint32_t n) { return (4u * n + 7u) & ~7u; }

  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    const uint32_t n = d.param;
    uint8_t *f = push(s, d.frame_bytes[0]);
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
    pop(s, f, d.frame_bytes[0]);
  }

  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t arg) {
    run_threads<ProgPaperScalars>(e, work, first, W, n, arg);
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
  static constexpr uint32_t kProgram = DSR_PROG_PAPER_ARRAYS;
  static constexpr bool kDense = false;
  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    uint8_t *f = push(s, d.frame_bytes[0]);
    if (!f) return;
    uint32_t *w = reinterpret_cast<uint32_t *>(f);
    for (uint32_t i = lane_id(); i < d.frame_bytes[0] / 4u; i += 32u) w[i] = 10u;
    __syncwarp();
    parallel<ProgPaperArrays>(e, 0, region_width(d), 0);
    pop(s, f, d.frame_bytes[0]);
  }

  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t arg) {
    run_threads<ProgPaperArrays>(e, work, first, W, n, arg);
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
// Scalars program: R = param sequential regions per team, each pushing int32 s[4]
// from image[r]; out[(r*T + team)*W' + tid] = (s0*tid + s1) ^
// ((s2 >> (tid & 7)) + s3). The master warp loads the frames of the next
// 32 regions while the current ones run (one region per lane).
// ---------------------------------------------------------------------------
struct ProgScalars {
  static constexpr uint32_t kProgram = DSR_PROG_SCALARS;
  static constexpr bool kDense = false;
  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    const uint32_t R = d.param, width = region_width(d), lane = lane_id();
    const uint4 *img = reinterpret_cast<const uint4 *>(e.images + d.image_offset);
    // lane l holds the frame of region (32 * batch + l): the loads for the
    // next batch are in flight while the current 32 regions run
    const uint4 zero = make_uint4(0, 0, 0, 0);
    uint4 cur = lane < R ? __ldg(img + lane) : zero;
    uint4 nxt = 32u + lane < R ? __ldg(img + 32u + lane) : zero;
    for (uint32_t r = 0; r < R; ++r) {
      const uint32_t l = r & 31u;
      if (l == 0 && r != 0) {
        cur = nxt;
        nxt = r + 32u + lane < R ? __ldg(img + r + 32u + lane) : zero;
      }
      uint4 v;
      v.x = __shfl_sync(0xffffffffu, cur.x, l);
      v.y = __shfl_sync(0xffffffffu, cur.y, l);
      v.z = __shfl_sync(0xffffffffu, cur.z, l);
      v.w = __shfl_sync(0xffffffffu, cur.w, l);
      uint8_t *f = push(s, 16);
      if (!f) return;
      if (lane == 0) *reinterpret_cast<uint4 *>(f) = v;
      __syncwarp();
      parallel<ProgScalars>(e, 0, width, r);
      pop(s, f, 16);
    }
  }

  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t arg) {
    run_threads<ProgScalars>(e, work, first, W, n, arg);
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t r) {
    const uint4 v = *reinterpret_cast<const uint4 *>(ctrl()->frames[0].ptr);
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset);
    o[(static_cast<uint64_t>(r) * e.d->teams + e.team) * n + tid] =
        (v.x * tid + v.y) ^ ((v.z >> (tid & 7u)) + v.w);
  }
};

// ---------------------------------------------------------------------------
// Nested program: D nested master-side calls. Level k pushes F_k = {int32 s[16];
// int32 arr[256]} filled from image[team][k-1] XOR mix32(team*8 + k), with
// F_k.s[0] ^= F_{k-1}.s[15] for k > 1, then forks:
//   k < D: F_k.arr[i] = mix32(F_k.arr[i] + i) for the worker's strided i;
//          after the join F_k.s[15] = sum(F_k.arr) (the workers add their
//          new words into s[15], which the master cleared before the fork);
//   k = D: out[e] = mix32(e ^ sum_m (F_m.arr[j & 255] ^ F_m.s[j & 15])),
//          e = team*E + j, for every j < E (E = param), each j by one
//          worker.
// On the way out chk[k-1] = F_k.s[15], then F_k is popped.
// ---------------------------------------------------------------------------
struct ProgNested {
  static constexpr uint32_t kProgram = DSR_PROG_NESTED;
  static constexpr bool kDense = true;
  enum : uint32_t { kUpdate = 0, kInner = 1 };

  // A frame in the slab is published to the workers as its byte offset in
  // shared memory with kSmemArg set (the parallel call's argument word);
  // otherwise the argument is the level k and the workers read the frame
  // table. kInner with kSmemArg: all D frames lie back to back from there.
  static constexpr uint32_t kSmemArg = 0x80000000u;
  // Every level's frame is 16 scalars and int32[256] (descriptors of this
  // program are checked to say so).
  static constexpr uint32_t kFrameBytes = 1088u;

  __device__ static void master(const Env &e, Stack &s) {
    const uint32_t D = e.d->depth;
    // all levels' images at once, into the slab slots the pushes will take
    // (from byte `x0` of shared memory on)
    const uint32_t x0 = kCtrlBytes + s.sp;
    if (stage(s, image(e, 1), D * 1088u)) {
      levels<true>(e, s, x0);
    } else {
      if (lane_id() == 0) prefetch_l2(image(e, 1), D * 1088u);
      levels<false>(e, s, x0);
    }
  }

  // The D levels. kStaged: the images were staged from x0 on, so level k's
  // frame takes the slab slot x0 + 1088 (k - 1) (pushes are in order and
  // the staged total fitted the slab) and is filled once its slot is keyed.
  template <bool kStaged>
  __device__ static void levels(const Env &e, Stack &s, uint32_t x0) {
    const dsr_region_desc &d = *e.d;
    const uint32_t D = d.depth;
    uint32_t carry = 0;  // c_{k-1}, the sum the previous level left in word 15
    for (uint32_t k = 1; k <= D; ++k) {
      bool sm;
      uint8_t *f = push(s, kFrameBytes, &sm);
      if (!f) return;
      const uint32_t off = static_cast<uint32_t>(f - dsr_smem);  // meaningful when sm
      if (kStaged) {
        if (!sm || off != x0 + (k - 1) * 1088u) {
          set_status(s, DSR_ERR_INVALID);  // not where staging put the image
          return;
        }
        if (k == 1) {
          // the staged images land together; key level 1's slot now and
          // the deeper levels' while level 1's region runs
          wait_staged(s);
          key_levels(dsr_smem + x0, 0, 1, e.team);
        }
      } else {
        fill<!kDense>(s, f, sm, image(e, k), 1088u, mix32(e.team * 8u + k));
      }
      if (s.status() != DSR_OK) return;
      uint32_t *w = reinterpret_cast<uint32_t *>(f);
      if (lane_id() == 0) {
        if (k > 1) w[0] ^= carry;
        // the workers of an update region add their new words into s[15]
        // (read by no region before the master sets it to the sum)
        if (k < D) w[15] = 0;
      }
      __syncwarp();
      // the last level's word 15 is final here (its region writes only the
      // output); earlier levels record their sums below
      if (k == D) set_chk(s, k - 1, w[15]);
      uint32_t arg = k;
      if (k < D && sm) arg = kSmemArg | off;
      if (kStaged && k == D) arg = kSmemArg | x0;
      fork<ProgNested>(e, k < D ? kUpdate : kInner, region_width(d), arg);
      // runtime work of the master: key the staged levels 2..D (frames not
      // pushed yet, slots the running region does not touch)
      if (kStaged && k == 1 && D > 1) key_levels(dsr_smem + x0, 1, D, e.team);
      join();
      if (k < D) {
        carry = w[15];  // the sum of arr the workers left there
        set_chk(s, k - 1, carry);
      }
    }
    for (uint32_t k = D; k >= 1; --k) {
      const uint8_t *p = kStaged ? dsr_smem + x0 + (k - 1) * 1088u : ctrl()->frames[k - 1].ptr;
      pop(s, p, kFrameBytes);
    }
  }

  // All D level images of the team (plain kernel, before the wait).
  __device__ static void prefetch_inputs(const Env &e) { prefetch_l2(image(e, 1), e.d->depth * 1088u); }

  // The image of level k of this team (1088 bytes).
  __device__ static const uint8_t *image(const Env &e, uint32_t k) {
    return e.images + e.d->image_offset +
           (static_cast<uint64_t>(e.team) * e.d->depth + (k - 1)) * 1088u;
  }

  // XOR level m's slot (1088 bytes from base + 1088 m) with
  // mix32(team*8 + m + 1), for the levels m0 <= m < m1 (master warp; the
  // key is computed once per level).
  __device__ static void key_levels(uint8_t *base, uint32_t m0, uint32_t m1, uint32_t team) {
    for (uint32_t m = m0; m < m1; ++m) {
      uint4 *v = reinterpret_cast<uint4 *>(base + m * kFrameBytes);
      const uint32_t key = mix32(team * 8u + m + 1u);
      for (uint32_t i = lane_id(); i < kFrameBytes / 16u; i += 32u) {
        uint4 x = v[i];
        x.x ^= key;
        x.y ^= key;
        x.z ^= key;
        x.w ^= key;
        v[i] = x;
      }
    }
    __syncwarp();
  }

  // Update regions: every worker updates its words of arr and adds the new
  // values up; a warp reduction and one shared-memory atomic per warp put
  // the frame's sum into s[15] (wrap-around adds: any order gives the sum
  // the master would take after the join). Every worker thread runs this,
  // so each warp's reduction has all its lanes.
  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t k) {
    if (work != kUpdate) {
      run_threads<ProgNested>(e, work, first, W, n, k);
      return;
    }
    uint32_t *f = k & kSmemArg ? reinterpret_cast<uint32_t *>(dsr_smem + (k & ~kSmemArg))
                               : reinterpret_cast<uint32_t *>(ctrl()->frames[k - 1].ptr);
    uint32_t *arr = f + 16, part = 0;
    for (uint32_t v = first; v < n; v += W)
      for (uint32_t i = v; i < 256u; i += n) {
        const uint32_t x = mix32(arr[i] + i);
        arr[i] = x;
        part += x;
      }
    part = warp_sum(part);
    if (lane_id() == 0 && part) atomicAdd(f + 15, part);
  }

  // The innermost region when E is a multiple of 256 and n >= 64, frames in
  // the slab. Summed over the levels, arr[j & 255] ^ s[j & 15] depends on
  // j & 255 alone (16 divides 256), so thread tid takes the groups of 4
  // elements of one class q = tid mod 64 (j0 & 255 = 4q): it sums the
  // class's 4 words over the levels once, then writes j0 = 4q + 256p for
  // its periods p = tid / 64, + P, + 2P, ... < E / 256, P being the number
  // of the region's threads in class q. Every element is written by one
  // thread, and a warp's 32 threads write 512 consecutive bytes.
  template <uint32_t kD>
  __device__ static void inner_cls(uint32_t base, uint32_t *o, uint32_t ebase, uint32_t tid,
                                   uint32_t n, uint32_t NP) {
    const uint32_t q = tid & 63u;
    const uint32_t P = (n - q + 63u) >> 6;  // threads t < n with t mod 64 == q
    const uint8_t *fs = dsr_smem + base;    // level 0's scalars; its array 64 bytes on
    const uint32_t oa = 64u + 16u * q, os = 16u * (q & 3u);
    uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (uint32_t m = 0; m < kD; ++m) {
      const uint4 a = *reinterpret_cast<const uint4 *>(fs + m * kFrameBytes + oa);
      const uint4 sv = *reinterpret_cast<const uint4 *>(fs + m * kFrameBytes + os);
      acc.x += a.x ^ sv.x;
      acc.y += a.y ^ sv.y;
      acc.z += a.z ^ sv.z;
      acc.w += a.w ^ sv.w;
    }
    const uint32_t p0 = tid >> 6;
    uint4 *dst = reinterpret_cast<uint4 *>(o) + q + (p0 << 6);
    uint32_t e0 = ebase + (q << 2) + (p0 << 8);
    for (uint32_t c = p0 < NP ? (NP - p0 + P - 1u) / P : 0u; c; --c) {
      uint4 r;
      r.x = mix32(e0 ^ acc.x);
      r.y = mix32((e0 | 1u) ^ acc.y);
      r.z = mix32((e0 | 2u) ^ acc.z);
      r.w = mix32((e0 | 3u) ^ acc.w);
      *dst = r;
      dst += P << 6;
      e0 += P << 8;
    }
  }

  // The innermost region (update regions run in run() above).
  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n, uint32_t k) {
    const uint32_t D = e.d->depth, E = e.d->param;
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset) +
                  static_cast<uint64_t>(e.team) * E;
    const uint32_t ebase = e.team * E;
    // Each element j is written by exactly one thread: by classes of 4 (the
    // frames in the slab, E a multiple of 256, 64 threads or more), or one
    // element j = tid, tid + n, ... at a time.
    if ((E & 255u) == 0 && n >= 64u && (k & kSmemArg)) {
      const uint32_t base = k & ~kSmemArg;
      switch (D) {
        case 1: inner_cls<1>(base, o, ebase, tid, n, E >> 8); return;
        case 2: inner_cls<2>(base, o, ebase, tid, n, E >> 8); return;
        case 3: inner_cls<3>(base, o, ebase, tid, n, E >> 8); return;
        default: inner_cls<4>(base, o, ebase, tid, n, E >> 8); return;
      }
    }
    for (uint32_t j = tid; j < E; j += n) {
      uint32_t acc = 0;
      for (uint32_t m = 0; m < D; ++m) {
        const uint32_t *f = frame_words(m);
        acc += f[16u + (j & 255u)] ^ f[j & 15u];
      }
      o[j] = mix32((ebase + j) ^ acc);
    }
  }
};

// ---------------------------------------------------------------------------
// Sweep program: one frame float arr[L] (L = frame_bytes/4) copied from
// image[team]; out[team*W' + tid] = arr[tid] + arr[tid + W'] + ... in index
// order, each addition rounded to fp32 (no contraction). A large frame in
// the slab is filled by a streamed fill (the region's argument is then 1):
// the workers sum each chunk as it lands.
// ---------------------------------------------------------------------------
struct ProgSweep {
  static constexpr uint32_t kProgram = DSR_PROG_SWEEP;
  static constexpr bool kDense = false;
  // The team's image (plain kernel, before the wait), for frames of up to
  // 32 KiB: a launch's larger images (up to 100 MB at 192 KiB) prefetched at
  // once contend with the fills and ran slower.
  __device__ static void prefetch_inputs(const Env &e) {
    const uint32_t S = e.d->frame_bytes[0];
    if (S <= 32768u)
      prefetch_l2(e.images + e.d->image_offset + static_cast<uint64_t>(e.team) * S, S & ~15u);
  }
  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    const uint32_t S = d.frame_bytes[0];
    bool sm;
    uint8_t *f = push(s, S, &sm);
    if (!f) return;
    const uint8_t *src = e.images + d.image_offset + static_cast<uint64_t>(e.team) * S;
    const bool streamed = sm && S >= kStreamMinBytes && fill_streamed(s, f, src, S);
    if (!streamed) {
      // a spilled frame's image is pulled towards L2 first, so the copy
      // across the workers meets fewer DRAM round trips
      if (!sm && lane_id() == 0) prefetch_l2(src, S & ~15u);
      fill<!kDense>(s, f, sm, src, S, 0u);
    }
    if (s.status() != DSR_OK) return;
    parallel<ProgSweep>(e, 0, region_width(d), streamed ? 1u : 0u);
    stream_finish(s);
    pop(s, f, S);
  }

  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t arg) {
    run_threads<ProgSweep>(e, work, first, W, n, arg);
  }

  __device__ static void body(const Env &e, uint32_t, uint32_t tid, uint32_t n,
                              uint32_t streamed) {
    const float *arr = reinterpret_cast<const float *>(ctrl()->frames[0].ptr);
    const uint32_t L = ctrl()->frames[0].bytes / 4u;
    // a spilled frame is read from L2/HBM: twice the loads in flight
    const float acc = __isShared(arr) ? strided_sum<16>(arr, L, tid, n, streamed)
                                      : strided_sum<32>(arr, L, tid, n, streamed);
    reinterpret_cast<float *>(e.out + e.d->out_offset)[e.team * n + tid] = acc;
  }

  // arr[tid] + arr[tid + n] + ... left to right in fp32. Rounds of kB loads
  // in flight (then of 4, then single loads), each followed by its
  // additions one by one in index order: the sum is the same left-to-right
  // fp32 sum, but the memory latency (shared memory, or L2/HBM for a
  // spilled frame) is paid once per round instead of once per element.
  template <uint32_t kB>
  __device__ static float strided_sum(const float *arr, uint32_t L, uint32_t tid, uint32_t n,
                                      uint32_t streamed) {
    float acc = 0.0f;
    uint32_t i = tid;
    // bytes of a streamed frame known to have landed (all of any other)
    uint32_t ready = streamed ? 0u : 0xffffffffu;
    sum_rounds<kB>(arr, L, n, i, acc, ready);
    sum_rounds<4>(arr, L, n, i, acc, ready);
    sum_rounds<1>(arr, L, n, i, acc, ready);
    return acc;
  }

  template <uint32_t kB>
  __device__ static void sum_rounds(const float *arr, uint32_t L, uint32_t n, uint32_t &i,
                                    float &acc, uint32_t &ready) {
    for (; i + (kB - 1u) * n < L; i += kB * n) {
      const uint32_t end = 4u * (i + (kB - 1u) * n) + 4u;  // past the round's last byte
      if (end > ready) ready = stream_ready(end, ready);
      float x[kB];
#pragma unroll
      for (uint32_t u = 0; u < kB; ++u) x[u] = arr[i + u * n];
#pragma unroll
      for (uint32_t u = 0; u < kB; ++u) acc = __fadd_rn(acc, x[u]);
    }
  }
};

// ---------------------------------------------------------------------------
// Hetero program (heterogeneous instances): D levels of F_k = int32[L_k] filled from the instance's level
// images XOR mix32(salt + team*8 + k), F_k[0] ^= c_{k-1} for k > 1, then:
//   k < D: F_k[w] = mix32(F_k[w] + w) for the worker's strided w; c_k =
//          sum of F_k (= chk[k-1]), added up by the workers as they update
//          it and read by the master after the join;
//   k = D: out[team*W' + tid] = sum over m <= D and the worker's strided w
//          of mix32(F_m[w] ^ (m << 24) ^ w).
// chk[D-1] = F_D[0]; the frames are popped in reverse order.
// ---------------------------------------------------------------------------
struct ProgHetero {
  static constexpr uint32_t kProgram = DSR_PROG_HETERO;
  static constexpr bool kDense = false;
  enum : uint32_t { kUpdate = 0, kInner = 1 };

  // The instance's level images (plain kernel, before the wait). Every team
  // reads the same images, so team 0 alone asks for them.
  __device__ static void prefetch_inputs(const Env &e) {
    if (e.team != 0) return;
    uint32_t total = 0;
    for (uint32_t k = 0; k < e.d->depth && k < DSR_MAX_DEPTH; ++k)
      total += (e.d->frame_bytes[k] + 15u) & ~15u;
    prefetch_l2(e.images + e.d->image_offset, total);
  }

  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    const uint32_t D = d.depth, width = region_width(d);
    const uint8_t *img = e.images + d.image_offset;
    uint32_t total = 0;
    for (uint32_t k = 0; k < D; ++k) total += (d.frame_bytes[k] + 15u) & ~15u;
    // every level's image at once, into the slab slots the pushes will take
    // (the images are laid out per level, 16-byte padded, as the slab is)
    uint8_t *expect = slab_base() + s.sp;
    const bool staged = stage(s, img, total);
    if (!staged && lane_id() == 0) prefetch_l2(img, total);
    uint32_t c_prev = 0;
    for (uint32_t k = 1; k <= D; ++k) {
      const uint32_t S = d.frame_bytes[k - 1];
      bool sm;
      uint8_t *f = push(s, S, &sm);
      if (!f) return;
      const uint32_t key = mix32(d.salt + e.team * 8u + k);
      if (staged && k == 1) wait_staged(s);
      if (staged && f == expect) {
        key_in_place(f, S, key);
        if (lane_id() == 0 && k > 1) reinterpret_cast<uint32_t *>(f)[0] ^= c_prev;
      } else {
        // F_k[0] ^= c_{k-1} applied by the thread that copies word 0
        fill<!kDense>(s, f, sm, img, S, key, k > 1 ? c_prev : 0u);
      }
      expect += (S + 15u) & ~15u;
      if (s.status() != DSR_OK) return;
      img += (S + 15u) & ~15u;
      if (lane_id() == 0) {
        // the update region's workers sum F_k here; the innermost region
        // gets the shared-memory offset of its accumulator (0: none)
        // (the persistent kernels' area after the slab, else the slab above
        // the frames when it has room)
        const uint32_t need = 4u * width, area = acc_area(s);
        ctrl()->acc = k < D || width < 4u ? 0u
                      : area ? area : (s.sp + need <= s.slab_bytes ? kCtrlBytes + s.sp : 0u);
      }
      __syncwarp();
      if (k == D) {
        // F_D[0], the last check word, is final now (the innermost region
        // only reads the frames): loaded before the fork, used after the join
        c_prev = reinterpret_cast<const uint32_t *>(f)[0];
      }
      parallel<ProgHetero>(e, k < D ? kUpdate : kInner, width, k);
      if (k < D) c_prev = ctrl()->acc;
      set_chk(s, k - 1, c_prev);
    }
    for (uint32_t k = D; k >= 1; --k) pop(s, ctrl()->frames[k - 1].ptr, d.frame_bytes[k - 1]);
  }

  // A thread's words w = v, v + n, ... < L of a frame: the sum of
  // mix32(F[w] ^ tag ^ w), in rounds of four and then two with the round's
  // loads issued before any of its hashing (a spilled frame's words are L2
  // round trips). Wrap-around sums: any order gives the same value.
  __device__ static uint32_t hash_words(const uint32_t *f, uint32_t v, uint32_t L, uint32_t n,
                                        uint32_t tag) {
    uint32_t acc = 0, w = v;
    for (; w + 3u * n < L; w += 4u * n) {
      const uint32_t x0 = f[w], x1 = f[w + n], x2 = f[w + 2u * n], x3 = f[w + 3u * n];
      acc += (mix32(x0 ^ tag ^ w) + mix32(x1 ^ tag ^ (w + n))) +
             (mix32(x2 ^ tag ^ (w + 2u * n)) + mix32(x3 ^ tag ^ (w + 3u * n)));
    }
    if (w + n < L) {
      const uint32_t x0 = f[w], x1 = f[w + n];
      acc += mix32(x0 ^ tag ^ w) + mix32(x1 ^ tag ^ (w + n));
      w += 2u * n;
    }
    if (w < L) acc += mix32(f[w] ^ tag ^ w);
    return acc;
  }

  // Update region: F[w] = mix32(F[w] + w) for every word, and the sum of
  // the new words. Each word's update stands alone, so the workers take the
  // frame by 16-byte vectors (vector i by worker i mod W, two vectors in
  // flight per round) instead of thread by thread: every word is updated
  // once, as the region's threads would, with many words in flight.
  __device__ static uint32_t update_frame(uint32_t *f, uint32_t L, uint32_t first, uint32_t W) {
    uint4 *f4 = reinterpret_cast<uint4 *>(f);  // frames are 16-byte aligned
    const uint32_t nv = L / 4u;
    uint32_t part = 0, i = first;
    for (; i + W < nv; i += 2u * W) {
      uint4 a = f4[i], b = f4[i + W];
      const uint32_t wa = 4u * i, wb = 4u * (i + W);
      a.x = mix32(a.x + wa);
      a.y = mix32(a.y + wa + 1u);
      a.z = mix32(a.z + wa + 2u);
      a.w = mix32(a.w + wa + 3u);
      b.x = mix32(b.x + wb);
      b.y = mix32(b.y + wb + 1u);
      b.z = mix32(b.z + wb + 2u);
      b.w = mix32(b.w + wb + 3u);
      f4[i] = a;
      f4[i + W] = b;
      part += (a.x + a.y) + (a.z + a.w) + (b.x + b.y) + (b.z + b.w);
    }
    if (i < nv) {
      uint4 a = f4[i];
      const uint32_t wa = 4u * i;
      a.x = mix32(a.x + wa);
      a.y = mix32(a.y + wa + 1u);
      a.z = mix32(a.z + wa + 2u);
      a.w = mix32(a.w + wa + 3u);
      f4[i] = a;
      part += (a.x + a.y) + (a.z + a.w);
    }
    for (uint32_t w = 4u * nv + first; w < L; w += W) {  // the last L mod 4 words
      const uint32_t y = mix32(f[w] + w);
      f[w] = y;
      part += y;
    }
    return part;
  }

  // Innermost region with a shared-memory accumulator of n words at byte
  // `acc_off`: out[v] = sum over the frames m and their words w with
  // w mod n == v of mix32(F_m[w] ^ (m+1) << 24 ^ w). The workers take each
  // frame by 16-byte vectors (vector i by worker i mod W) and add each word's
  // hash into acc[w mod n] with a shared-memory atomic; two barriers of the
  // workers alone (named barrier 3) separate clearing, adding and writing
  // out. Wrap-around adds: the same sums as each thread's own loop.
  // acc[(w + c) mod n] += mix32(x.c ^ tag ^ (w + c)) for the 4 words of a
  // vector starting at word w, r = w mod n.
  __device__ static void add_vec(uint32_t *acc, const uint4 x, uint32_t w, uint32_t tag,
                                 uint32_t r, uint32_t n) {
    uint32_t r1 = r + 1u, r2 = r + 2u, r3 = r + 3u;
    r1 = r1 >= n ? r1 - n : r1;
    r2 = r2 >= n ? r2 - n : r2;
    r3 = r3 >= n ? r3 - n : r3;
    atomicAdd(acc + r, mix32(x.x ^ tag ^ w));
    atomicAdd(acc + r1, mix32(x.y ^ tag ^ (w + 1u)));
    atomicAdd(acc + r2, mix32(x.z ^ tag ^ (w + 2u)));
    atomicAdd(acc + r3, mix32(x.w ^ tag ^ (w + 3u)));
  }

  __device__ static void inner_acc(const Env &e, uint32_t first, uint32_t W, uint32_t n,
                                   uint32_t D, uint32_t acc_off) {
    const Ctrl *c = ctrl();
    uint32_t *acc = reinterpret_cast<uint32_t *>(dsr_smem + acc_off);
    for (uint32_t v = first; v < n; v += W) acc[v] = 0u;
    named_bar(kWorkerBar, W);
    const uint32_t step = (4u * W) % n;  // n >= 4
    for (uint32_t m = 0; m < D; ++m) {
      const uint32_t *f = reinterpret_cast<const uint32_t *>(c->frames[m].ptr);
      const uint32_t L = c->frames[m].bytes / 4u, nv = L / 4u, tag = (m + 1u) << 24;
      const uint4 *f4 = reinterpret_cast<const uint4 *>(f);
      uint32_t r = (4u * first) % n;  // (4 i) mod n for this worker's vector i
      if ((n & 3u) == 0) {
        // r is then a multiple of 4 below n: its vector's 4 outputs are
        // r .. r + 3, none past n
        for (uint32_t i = first; i < nv; i += W) {
          const uint4 x = f4[i];
          const uint32_t tw = tag ^ (4u * i);  // 4i + c == 4i ^ c for c < 4
          atomicAdd(acc + r, mix32(x.x ^ tw));
          atomicAdd(acc + r + 1u, mix32(x.y ^ tw ^ 1u));
          atomicAdd(acc + r + 2u, mix32(x.z ^ tw ^ 2u));
          atomicAdd(acc + r + 3u, mix32(x.w ^ tw ^ 3u));
          r += step;
          r = r >= n ? r - n : r;
        }
      } else {
        for (uint32_t i = first; i < nv; i += W) {
          add_vec(acc, f4[i], 4u * i, tag, r, n);
          r += step;
          r = r >= n ? r - n : r;
        }
      }
      for (uint32_t w = 4u * nv + first; w < L; w += W) atomicAdd(acc + w % n, mix32(f[w] ^ tag ^ w));
    }
    named_bar(kWorkerBar, W);
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset) +
                  static_cast<uint64_t>(e.team) * n;
    for (uint32_t v = first; v < n; v += W) o[v] = acc[v];
  }

  // The worker's virtual threads with the frame pointers and sizes read
  // once per region instead of once per thread. An update region also sums
  // the frame's new words: per worker, then per warp (a reduction), then
  // one shared-memory atomic per warp into the control block (wrap-around
  // adds, so the order does not matter); every worker thread runs this, so
  // each warp's reduction has all its lanes.
  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t k) {
    Ctrl *c = ctrl();
    if (work == kUpdate) {
      uint32_t part = update_frame(reinterpret_cast<uint32_t *>(c->frames[k - 1].ptr),
                                   c->frames[k - 1].bytes / 4u, first, W);
      part = warp_sum(part);
      if (lane_id() == 0 && part) atomicAdd(&c->acc, part);
      return;
    }
    if (const uint32_t acc_off = c->acc) {
      inner_acc(e, first, W, n, k, acc_off);
      return;
    }
    const uint32_t *f[DSR_MAX_DEPTH];
    uint32_t L[DSR_MAX_DEPTH];
#pragma unroll
    for (uint32_t m = 0; m < DSR_MAX_DEPTH; ++m) {
      f[m] = m < k ? reinterpret_cast<const uint32_t *>(c->frames[m].ptr) : nullptr;
      L[m] = m < k ? c->frames[m].bytes / 4u : 0u;
    }
    uint32_t *o = reinterpret_cast<uint32_t *>(e.out + e.d->out_offset) +
                  static_cast<uint64_t>(e.team) * n;
    // threads at or past every frame's end have no elements: their sum is 0
    const uint32_t Lmax = max(max(L[0], L[1]), max(L[2], L[3]));
    uint32_t v = first;
    for (; v < n && v < Lmax; v += W) {
      uint32_t acc = 0;
#pragma unroll
      for (uint32_t m = 0; m < DSR_MAX_DEPTH; ++m)
        if (m < k) acc += hash_words(f[m], v, L[m], n, (m + 1u) << 24);
      o[v] = acc;
    }
    for (; v < n; v += W) o[v] = 0u;
  }

};

// ---------------------------------------------------------------------------
// Worker-level sharing (Sec. 7, future work: sharing among workers, an
// all-to-all pattern that needs far more stack, with a runtime-managed
// global stack behind the shared one). The master pushes F = int32 s[4]
// from the team's image and forks. Every worker t < W' is then itself the
// master of a nested parallel region: it pushes G_t = int32[L] on a stack
// of its own warp, G_t[i] = base[i] ^ mix32(s0 + t), and its nested team
// -- the 32 lanes of its warp, the mapping of CUDA-NP (Sec. 2) -- runs
// G_t[w] = mix32(G_t[w] + s1 + w); afterwards out[team*W' + t] =
// (sum G_t) ^ s2. After the join the master stores chk[0] = sum of the
// team's outputs and pops F.
//
// Warp stacks. What the team's slab and overflow slab have left after F is
// split evenly (16-byte units) over the W/32 worker warps. A warp pushes
// its lanes' frames in lane order, first fit (its slab share, else its
// overflow share); a frame that fits neither makes the team OVERFLOW and
// that worker (and the warp's later ones, whose frames fit no better) runs
// nothing. The frames stay live until the warp's last nested region has
// run, then are popped in reverse order. The stack pointers never leave
// registers: every frame has the same size, so lane l's slot follows from
// l. A frame's slot reaches the lanes of the nested team by a warp shuffle
// (the frame table of the warp is a register per lane).
// ---------------------------------------------------------------------------
// kSmemShare: the nested teams get their workers' keys and frame-slot
// offsets from a per-warp table in shared memory (each worker writes its
// entry, __syncwarp, the lanes read the entry they need) instead of by warp
// shuffles; the same results, for measuring the two ways of sharing within
// a warp (a descriptor's param selects it in the plain launch).
template <bool kSmemShare>
struct ProgWorkersT {
  static constexpr uint32_t kProgram = DSR_PROG_WORKERS;
  static constexpr bool kDense = false;
  // Teams hold large warp stacks, so few fit an SM: the plain kernel gets
  // a register budget for half the usual resident CTAs.
  static constexpr bool kWideRegs = true;

  __device__ static const uint8_t *image(const Env &e) {
    const dsr_region_desc &d = *e.d;
    return e.images + d.image_offset +
           static_cast<uint64_t>(e.team) * (16u + ((d.frame_bytes[1] + 15u) & ~15u));
  }

  __device__ static void master(const Env &e, Stack &s) {
    const dsr_region_desc &d = *e.d;
    uint8_t *F = push(s, 16);
    if (!F) return;
    if (lane_id() == 0)
      *reinterpret_cast<uint4 *>(F) = __ldg(reinterpret_cast<const uint4 *>(image(e)));
    // the warp stacks' shares of what the team's stack has left
    const uint32_t nwarps = team_workers() / 32u;
    const uint64_t ovf_left = ctrl()->ovf_bytes - s.gsp;
    if (lane_id() == 0) {
      Ctrl *c = ctrl();
      c->wstack_off = kCtrlBytes + s.sp;
      c->wslab = ((s.slab_bytes - s.sp) / nwarps) & ~15u;
      c->wovf = c->ovf ? c->ovf + s.gsp : nullptr;
      c->wovf_bytes = c->ovf ? (ovf_left / nwarps) & ~15ull : 0ull;
      c->whwm = 0;
      c->wspill = 0;
      c->wfail = 0;
    }
    __syncwarp();
    const uint32_t width = region_width(d);
    parallel<ProgWorkersT>(e, 0, width, 0);
    const Ctrl *c = ctrl();
    s.hwm += c->whwm;
    s.spill += c->wspill;
    if (c->wfail) set_status(s, DSR_ERR_OVERFLOW);
    // the workers' outputs, read by the master after the join
    const uint32_t *o = reinterpret_cast<const uint32_t *>(e.out + d.out_offset) +
                        static_cast<uint64_t>(e.team) * width;
    uint32_t v = 0;
    for (uint32_t t = lane_id(); t < width; t += 32u) v += o[t];
    set_chk(s, 0, warp_sum(v));
    pop(s, F, 16);
  }

  // The warp's work is done in three phases, each over all of its workers'
  // frames at once and separated by __syncwarp: the workers' fills, then
  // every worker's nested region, then each worker's sum, by its own lane.
  // A phase walks the (frame, element) pairs of a run of frames with the
  // warp's 32 lanes side by side (Walk), so per-frame overhead is paid once
  // per warp rather than once per frame. In the nested phase the nested
  // regions of the warp's workers run concurrently, each word once, as any
  // schedule of their teams may; the fill moves 16-byte vectors and the
  // nested region single words, so the data crosses lanes through the
  // frames. The workers publish their keys and their frames' slot offsets
  // to the lanes that use them by shuffles.
  struct Walk {  // element idx = lane + 32 i of frames l0, l0 + 1, ... (cnt each)
    uint32_t l, q, dl, dq, cnt;
    __device__ Walk(uint32_t l0, uint32_t cnt_) : cnt(cnt_) {
      const uint32_t lane = lane_id();
      l = l0 + lane / cnt;
      q = lane % cnt;
      dl = 32u / cnt;
      dq = 32u % cnt;
    }
    __device__ void next() {
      q += dq;
      l += dl;
      if (q >= cnt) {
        q -= cnt;
        ++l;
      }
    }
  };

  // Fill of frames l0 .. l1-1 stored back to back (stride fp) from `base`:
  // G_l = image words ^ key of worker l (key_lane: this lane's worker's key).
  // The key of worker l of the warp (this lane's is key_lane): by shuffle,
  // or from the warp's table in shared memory.
  __device__ static uint32_t key_of(uint32_t key_lane, const uint32_t *tab, uint32_t l) {
    if constexpr (kSmemShare) return tab[l];
    return __shfl_sync(0xffffffffu, key_lane, l);
  }
  __device__ static uint32_t off_of(uint32_t off_lane, const uint32_t *tab, uint32_t l) {
    if constexpr (kSmemShare) return tab[32u + l];
    return __shfl_sync(0xffffffffu, off_lane, l);
  }

  template <bool kSmem>
  __device__ static void fill_phase(uint8_t *base, uint32_t fp, uint32_t l0, uint32_t l1,
                                    uint32_t L, const uint4 *img4, uint32_t key_lane,
                                    const uint32_t *tab) {
    const uint32_t nv = L / 4u, tw = L - 4u * nv;
    if (nv) {
      const uint32_t total = (l1 - l0) * nv;
      Walk it(l0, nv);
      for (uint32_t i = lane_id(); i < ((total + 31u) & ~31u); i += 32u, it.next()) {
        const uint32_t key = key_of(key_lane, tab, it.l & 31u);
        if (i < total) {
          uint4 x = __ldg(img4 + it.q);
          x.x ^= key;
          x.y ^= key;
          x.z ^= key;
          x.w ^= key;
          reinterpret_cast<uint4 *>(base + (it.l - l0) * fp)[it.q] = x;
        }
      }
    }
    if (tw) {  // the last L % 4 words of each frame
      const uint32_t total = (l1 - l0) * tw;
      const uint32_t *imgw = reinterpret_cast<const uint32_t *>(img4) + 4u * nv;
      Walk it(l0, tw);
      for (uint32_t i = lane_id(); i < ((total + 31u) & ~31u); i += 32u, it.next()) {
        const uint32_t key = key_of(key_lane, tab, it.l & 31u);
        if (i < total)
          reinterpret_cast<uint32_t *>(base + (it.l - l0) * fp)[4u * nv + it.q] =
              __ldg(imgw + it.q) ^ key;
      }
    }
  }

  // Nested regions of frames l0 .. l1-1: G_l[w] = mix32(G_l[w] + s1 + w).
  // off_lane: this lane's worker's slot offset from `base`.
  // Four steps of the walk at a time, their loads issued before any of
  // their stores (the words are distinct), so the latency of a spilled
  // frame's words is paid once per four.
  template <bool kSmem>
  __device__ static void nested_phase(uint8_t *base, uint32_t l0, uint32_t l1, uint32_t L,
                                      uint32_t s1, uint32_t off_lane, const uint32_t *tab) {
    constexpr uint32_t kB = 4;
    if ((L & 31u) == 0) {
      // L a multiple of 32: the frames lie back to back (a frame's slot is
      // exactly 4 L bytes) and each step of the lanes covers 32 consecutive
      // words of one frame, so a counter gives each word's index in its
      // frame, and no slot offset or walk is needed
      uint32_t *p = reinterpret_cast<uint32_t *>(base) + lane_id();
      const uint32_t rows = (l1 - l0) * (L >> 5);
      uint32_t w = lane_id();  // index in its frame of this lane's word of row r
      for (uint32_t r = 0; r < rows; r += kB) {
        uint32_t v[kB], ww[kB];
#pragma unroll
        for (uint32_t u = 0; u < kB; ++u) {
          ww[u] = w;
          v[u] = r + u < rows ? p[32u * (r + u)] : 0u;
          w += 32u;
          if (w >= L) w -= L;
        }
#pragma unroll
        for (uint32_t u = 0; u < kB; ++u)
          if (r + u < rows) p[32u * (r + u)] = mix32(v[u] + s1 + ww[u]);
      }
      return;
    }
    const uint32_t total = (l1 - l0) * L;
    Walk it(l0, L);
    for (uint32_t i = lane_id(); i < ((total + 32u * kB - 1u) & ~(32u * kB - 1u));
         i += 32u * kB) {
      uint32_t *g[kB];
      uint32_t v[kB], w[kB];
#pragma unroll
      for (uint32_t u = 0; u < kB; ++u) {
        const uint32_t off = off_of(off_lane, tab, it.l & 31u);
        g[u] = i + 32u * u < total ? reinterpret_cast<uint32_t *>(base + off) + it.q : nullptr;
        w[u] = it.q;
        v[u] = g[u] ? *g[u] : 0u;
        it.next();
      }
#pragma unroll
      for (uint32_t u = 0; u < kB; ++u)
        if (g[u]) *g[u] = mix32(v[u] + s1 + w[u]);
    }
  }

  // A worker's sum of its own frame (its lane alone), the vectors read in
  // an order rotated by the lane so that lanes meet different banks.
  __device__ static uint32_t frame_sum_own(const uint8_t *g, uint32_t L) {
    const uint32_t nv = L / 4u;
    const uint4 *g4 = reinterpret_cast<const uint4 *>(g);
    uint32_t part = 0, q = nv ? lane_id() % nv : 0u;
#pragma unroll 4
    for (uint32_t k = 0; k < nv; ++k) {
      const uint4 x = g4[q];
      part += x.x + x.y + x.z + x.w;
      q = q + 1u == nv ? 0u : q + 1u;
    }
    const uint32_t *gw = reinterpret_cast<const uint32_t *>(g);
    for (uint32_t w = 4u * nv; w < L; ++w) part += gw[w];
    return part;
  }

  // Every worker thread calls run() once (the region is no wider than the
  // workers); the warp is the unit of work.
  __device__ static void run(const Env &e, uint32_t, uint32_t tid, uint32_t, uint32_t n,
                             uint32_t) {
    const uint32_t lane = lane_id(), warp = tid >> 5, t0 = warp << 5;
    if (t0 >= n) return;  // no worker of this warp takes part (uniform in the warp)
    const uint32_t lanes = min(32u, n - t0);  // workers t0 .. t0 + lanes - 1
    Ctrl *c = ctrl();
    const dsr_region_desc &d = *e.d;
    const uint32_t L = d.frame_bytes[1] / 4u;
    const uint32_t fp = (d.frame_bytes[1] + 15u) & ~15u;
    // this warp's stack: lane order, first fit into the slab share, then
    // the overflow share
    const uint32_t in_slab = min(lanes, c->wslab / fp);
    const uint64_t ovf_fit = c->wovf_bytes / fp;
    const uint32_t pushed =
        static_cast<uint32_t>(min(static_cast<uint64_t>(lanes), in_slab + ovf_fit));
    if (lane == 0) {
      atomicAdd(&c->whwm, pushed * fp);
      atomicAdd(&c->wspill, (pushed - min(pushed, in_slab)) * fp);
      if (pushed < lanes) atomicOr(&c->wfail, 1u);
    }
    uint8_t *sbase = dsr_smem + c->wstack_off + warp * c->wslab;  // slab share
    uint8_t *gbase = c->wovf + warp * c->wovf_bytes;               // overflow share
    const uint32_t *F = reinterpret_cast<const uint32_t *>(c->frames[0].ptr);
    const uint32_t s0 = F[0], s1 = F[1], s2 = F[2];
    const uint4 *img4 = reinterpret_cast<const uint4 *>(image(e) + 16);
    // each worker's key and its frame's slot offset in its share
    const uint32_t key = mix32(s0 + t0 + lane);
    const uint32_t off = lane < in_slab ? lane * fp : (lane - in_slab) * fp;
    const uint32_t *tab = nullptr;
    if constexpr (kSmemShare) {
      // the warp's table: key of worker l at [l], its slot offset at [32 + l]
      __shared__ uint32_t share[DSR_MAX_THREADS / 32][64];
      share[warp][lane] = key;
      share[warp][32u + lane] = off;
      __syncwarp();
      tab = share[warp];
    }
    // the workers' sequential parts: their fills (order-free word copies)
    fill_phase<true>(sbase, fp, 0, in_slab, L, img4, key, tab);
    if (pushed > in_slab) fill_phase<false>(gbase, fp, in_slab, pushed, L, img4, key, tab);
    __syncwarp();  // fork of the nested regions
    nested_phase<true>(sbase, 0, in_slab, L, s1, off, tab);
    if (pushed > in_slab) nested_phase<false>(gbase, in_slab, pushed, L, s1, off, tab);
    __syncwarp();  // join
    if (lane < pushed) {
      const uint32_t sum = lane < in_slab ? frame_sum_own(sbase + off, L)
                                          : frame_sum_own(gbase + off, L);
      reinterpret_cast<uint32_t *>(e.out + d.out_offset)[static_cast<uint64_t>(e.team) * n + t0 +
                                                          lane] = sum ^ s2;
    }
    // the warp's frames are popped in reverse order: with register stack
    // pointers that is the end of the region
  }

  __device__ static void body(const Env &, uint32_t, uint32_t, uint32_t, uint32_t) {}
};

using ProgWorkers = ProgWorkersT<false>;
using ProgWorkersSmem = ProgWorkersT<true>;

}  // namespace dsr
