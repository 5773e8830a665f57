// parem_scan.cuh -- sm_103a kernels of the chunked speculative DFA scan.
//
// Mapping of Algorithm 1 onto the GPU
//   * Domain decomposition: the text is cut into rows ("segments") of S bytes; 32
//     consecutive rows form a chunk, owned by one warp, one row per lane.  Chunks are
//     taken in order from an atomic ticket counter by persistent warps.
//   * Candidate speculation (R = S n L): for row r > 0 the candidates are img(c), the
//     distinct states reachable on the class c of the byte that ends row r-1, minus the
//     dead state (a dead run needs no simulation).  Row 0 starts from q0 exactly.
//   * Candidate runs: the warp runs the candidates of one row in lockstep, one candidate per
//     lane register, and merges lanes whose states meet (__match_any_sync, or a per-warp
//     owner table when there are more than 32 candidates).  Once one live state is left
//     the row's map is constant from that offset t on; the lane that owns the row then runs
//     that single state over the rest of its row out of shared memory, where a TMA pipeline
//     stages 32 rows x 128 bytes per step (128-byte swizzle, conflict-free reads).
//   * Reduction / join: each chunk publishes its end state (MAPPED), then its match count
//     and dead flag given the end state of the previous chunk (AGGREGATE), then the prefix
//     (INCLUSIVE), found by a decoupled look-back over 32 predecessors at a time.  A row
//     whose candidates never merge keeps a full slot map (end, count per candidate).
//   * The matches inside [0, t) of each row are counted by re-running that prefix from the
//     resolved start; the same re-run checks that the start reaches the merged state.
//   * Emit pass: rows with matches are re-run from their resolved start and their positions
//     are written at the row's offset in the global order.
#pragma once

#include <cstdint>

#include "parem_internal.h"

namespace parem {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint4 ldg16(const uint8_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t ldg8(const uint8_t* p) {
  uint16_t v;
  asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t byte_of(const uint4& v, int i) {
  const uint32_t w = (i < 4) ? v.x : (i < 8) ? v.y : (i < 12) ? v.z : v.w;
  return (w >> (8 * (i & 3))) & 0xFFu;
}

__device__ __forceinline__ void set_error(DevResult* r, uint32_t code) {
  atomicCAS(&r->error, 0u, code);
}

__device__ __forceinline__ uint32_t read_error(const DevResult* r) {
  return *reinterpret_cast<const volatile uint32_t*>(&r->error);
}

// ---------------------------------------------------------------------------------------
// Transition table access.  LAYOUT kByteSmem: row = 256 byte columns; kClassSmem: row =
// class columns (byte -> column offset from colmap in smem); kClassGlobal: same in global
// memory (read through the read-only path, L2 resident).
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
struct Tab {
  const uint8_t* sm;       // dynamic smem base (aligned)
  uint32_t table_off;      // smem offset of the table
  uint32_t colmap_off;     // smem offset of the 256-entry column map
  const uint8_t* gtable;   // global table (kClassGlobal)
  uint32_t rowbytes;

  __device__ __forceinline__ uint32_t col(uint32_t b) const {
    if (LAYOUT == kByteSmem) return b * ESIZE;
    return reinterpret_cast<const uint32_t*>(sm + colmap_off)[b];
  }
  __device__ __forceinline__ uint32_t next(uint32_t s, uint32_t c) const {
    const uint32_t o = s * rowbytes + c;
    if (LAYOUT == kClassGlobal) {
      return ESIZE == 1 ? (uint32_t)__ldg(gtable + o)
                        : (uint32_t)__ldg(reinterpret_cast<const uint16_t*>(gtable + o));
    }
    return ESIZE == 1 ? (uint32_t)sm[table_off + o]
                      : (uint32_t)*reinterpret_cast<const uint16_t*>(sm + table_off + o);
  }
};

// Run [0, len) of a 16-byte aligned global range from state x.  Adds the matches to *cnt
// and returns the end state; stops early (returning dead) once the run is dead.
template <int LAYOUT, int ESIZE>
__device__ uint32_t run_range16(const Tab<LAYOUT, ESIZE>& tab, const uint8_t* p, uint64_t len,
                                uint32_t x, uint32_t dead, uint32_t first_accept, uint32_t* cnt) {
  uint32_t c = 0;
  for (uint64_t o = 0; o < len; o += 16) {
    const uint4 v = ldg16(p + o);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      x = tab.next(x, tab.col(byte_of(v, i)));
      c += (x >= first_accept);
    }
    if (x == dead) break;
  }
  // a dead run cannot have counted matches after dying (dead < first_accept)
  *cnt += c;
  return x;
}

// Run an arbitrary (unaligned) global byte range [0, len) from x, byte by byte.
template <int LAYOUT, int ESIZE>
__device__ uint32_t run_bytes(const Tab<LAYOUT, ESIZE>& tab, const uint8_t* p, uint64_t len,
                              uint32_t x, uint32_t dead, uint32_t first_accept, uint32_t* cnt) {
  uint32_t c = 0;
  for (uint64_t o = 0; o < len; ++o) {
    x = tab.next(x, tab.col(ldg8(p + o)));
    c += (x >= first_accept);
    if (x == dead) break;
  }
  *cnt += c;
  return x;
}

// Associative join of (dead, count) pairs in text order: everything after a death counts 0.
struct Pfx {
  uint32_t dead;
  uint64_t count;
};
__device__ __forceinline__ Pfx pfx_op(Pfx a, Pfx b) {  // a before b
  Pfx r;
  r.dead = a.dead | b.dead;
  r.count = a.dead ? a.count : a.count + b.count;
  return r;
}

__device__ __forceinline__ unsigned long long pack_status(uint32_t flag, uint32_t dead, uint32_t E,
                                                          uint64_t cnt) {
  return ((unsigned long long)flag << 62) | ((unsigned long long)(dead & 1u) << 61) |
         ((unsigned long long)(E & 0xFFFFu) << 45) | (cnt & kCountMask);
}

// Bounded wait on a stage barrier.  Returns false on timeout or when another warp failed.
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity, uint64_t budget,
                                           const DevResult* res) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if ((uint64_t)(clock64() - t0) > budget || read_error(res)) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Pass 1: speculation, main run, look-back.  P = candidate registers per lane.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE, int P>
__global__ void __launch_bounds__(1024, 1)
    k_spec_scan(const __grid_constant__ CUtensorMap tmap, const ScanParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const DeviceDfa& D = p.dfa;

  // stage the column map and (smem layouts) the table
  {
    const uint4* src = reinterpret_cast<const uint4*>(D.colmap);
    uint4* dst = reinterpret_cast<uint4*>(sm + p.smem_colmap_off);
    for (uint32_t i = threadIdx.x; i < 1024 / 16; i += blockDim.x) dst[i] = src[i];
    if (LAYOUT != kClassGlobal) {
      const uint4* ts = reinterpret_cast<const uint4*>(D.table);
      uint4* td = reinterpret_cast<uint4*>(sm + p.smem_table_off);
      for (uint32_t i = threadIdx.x; i < D.table_bytes / 16; i += blockDim.x) td[i] = ts[i];
    }
  }
  const uint32_t stage0 = p.smem_stage_off + warp * (kStages * kStageBytes);
  const uint32_t bar0 = p.smem_bar_off + warp * (kStages * 8);
  uint32_t* hash = reinterpret_cast<uint32_t*>(sm + p.smem_hash_off) + warp * kHashSize;
  if (lane == 0) {
    for (uint32_t s = 0; s < kStages; ++s) mbar_init(smem_u32(sm + bar0 + 8 * s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.table_off = p.smem_table_off;
  tab.colmap_off = p.smem_colmap_off;
  tab.gtable = D.table;
  tab.rowbytes = D.rowbytes;
  const uint32_t dead = D.dead;  // kEmpty when the DFA has no dead state
  const uint32_t A = D.first_accept;
  const uint32_t nblk = (uint32_t)(p.S / kBox);
  const uint32_t issue_first = nblk < kStages ? nblk : kStages;
  uint32_t phase_bits = 0;  // expected parity of each stage barrier
  uint32_t pending = 0;     // stages issued and not yet waited

  for (;;) {
    uint32_t ticket = 0;
    if (lane == 0) ticket = read_error(p.result) ? 0xFFFFFFFFu : atomicAdd(p.ticket, 1u);
    ticket = __shfl_sync(kFull, ticket, 0);
    if ((uint64_t)ticket >= p.n_chunks) break;
    const uint64_t j = ticket;
    const uint64_t row0 = j * kLanes;
    const uint64_t myrow = row0 + lane;
    const bool active = myrow < p.R;
    const uint32_t nrows = (uint32_t)((p.R - row0) < kLanes ? (p.R - row0) : kLanes);
    const uint8_t* body = p.text + p.h;  // 16-byte aligned

    // 1. start the TMA pipeline for this chunk
    if (lane == 0) {
      for (uint32_t b = 0; b < issue_first; ++b) {
        const uint32_t bar = smem_u32(sm + bar0 + 8 * b);
        mbar_arrive_expect_tx(bar, kStageBytes);
        tma_load_2d(smem_u32(sm + stage0 + b * kStageBytes), &tmap, bar, (int32_t)(b * kBox),
                    (int32_t)row0);
      }
    }
    pending |= (1u << issue_first) - 1u;
    bool failed = false;

    // 2. speculation, one row at a time, candidates across the lanes
    uint32_t my_t = 0, my_sigma = kEmpty, my_conv = 1, head_cnt = 0;
    const uint32_t cap = p.spec_cap;
    for (uint32_t k = 0; k < nrows && !failed; ++k) {
      const uint64_t r = row0 + k;
      if (r == 0) {
        // row 0 starts from the exact state: the initial state run over the head bytes
        uint32_t c0 = 0;
        const uint32_t sh = run_bytes(tab, p.text, p.h, p.init_state, dead, A, &c0);
        if (lane == 0) {
          my_t = 0;
          my_sigma = sh;
          my_conv = 1;
          head_cnt = c0;
        }
        continue;
      }
      const uint32_t cls = p.enum_all ? D.n_classes : (uint32_t)D.byte_class[ldg8(body + r * p.S - 1)];
      const uint32_t off = D.img_off[cls];
      const uint32_t m = D.img_off[cls + 1] - off;
      if (m <= 1 || m > 32u * P) {
        if (lane == k) {
          my_t = 0;
          my_conv = m <= 1;
          my_sigma = m == 1 ? (uint32_t)D.img[off] : dead;
          if (m > 32u * P) my_t = (uint32_t)p.S;
        }
        continue;
      }
      uint32_t st[P];
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const uint32_t slot = (uint32_t)i * 32u + lane;
        st[i] = slot < m ? (uint32_t)D.img[off + slot] : kEmpty;
      }
      const uint8_t* rowp = body + r * p.S;
      uint32_t pos = 0, sigma = kEmpty;
      bool conv = false;
      while (pos < cap) {
        uint4 v;
        if (pos < kStages * kBox) {
          const uint32_t b = pos / kBox;
          if (!stage_wait(smem_u32(sm + bar0 + 8 * b), (phase_bits >> b) & 1u, p.wait_budget,
                          p.result)) {
            set_error(p.result, kErrTimeout);
            failed = true;
            break;
          }
          const uint32_t ch = ((pos % kBox) / 16u) ^ (k & 7u);
          v = *reinterpret_cast<const uint4*>(sm + stage0 + b * kStageBytes + k * kBox + ch * 16u);
        } else {
          v = ldg16(rowp + pos);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int i2 = 0; i2 < 4; ++i2) {
            const uint32_t c = tab.col(byte_of(v, q * 4 + i2));
#pragma unroll
            for (int i = 0; i < P; ++i) {
              if (st[i] != kEmpty) {
                const uint32_t s2 = tab.next(st[i], c);
                st[i] = (s2 == dead) ? kEmpty : s2;
              }
            }
          }
          // merge lanes whose candidates met
          if (P == 1) {
            const unsigned grp = __match_any_sync(kFull, st[0]);
            if (st[0] != kEmpty && (uint32_t)(__ffs(grp) - 1) != lane) st[0] = kEmpty;
          } else {
#pragma unroll
            for (int i = 0; i < P; ++i)
              if (st[i] != kEmpty) hash[st[i] & (kHashSize - 1)] = (st[i] << 8) | ((uint32_t)i * 32u + lane);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < P; ++i) {
              if (st[i] != kEmpty) {
                const uint32_t e = hash[st[i] & (kHashSize - 1)];
                if ((e >> 8) == st[i] && (e & 0xFFu) != (uint32_t)i * 32u + lane) st[i] = kEmpty;
              }
            }
            __syncwarp();
          }
        }
        pos += 16;
        uint32_t live = 0, holder_reg = 0, holder_mask = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const unsigned b = __ballot_sync(kFull, st[i] != kEmpty);
          if (b && !holder_mask) {
            holder_mask = b;
            holder_reg = (uint32_t)i;
          }
          live += __popc(b);
        }
        if (live <= 1) {
          conv = true;
          if (live == 0) {
            sigma = dead;
          } else {
            uint32_t val = kEmpty;
#pragma unroll
            for (int i = 0; i < P; ++i)
              if ((uint32_t)i == holder_reg) val = st[i];
            sigma = __shfl_sync(kFull, val, __ffs(holder_mask) - 1);
          }
          break;
        }
      }
      if (lane == k) {
        my_conv = conv;
        my_t = conv ? pos : (uint32_t)p.S;
        my_sigma = sigma;
      }
    }

    // 3. slot maps of rows whose candidates did not merge (rare): every candidate runs
    //    the whole row (and the tail on the last row), lanes over candidates
    unsigned nonconv = __ballot_sync(kFull, active && !my_conv);
    while (nonconv && !failed) {
      const uint32_t k = __ffs(nonconv) - 1;
      nonconv &= nonconv - 1;
      const uint64_t r = row0 + k;
      const uint32_t cls = p.enum_all ? D.n_classes : (uint32_t)D.byte_class[ldg8(body + r * p.S - 1)];
      const uint32_t off = D.img_off[cls];
      const uint32_t m = D.img_off[cls + 1] - off;
      for (uint32_t base = 0; base < m; base += 32) {
        const uint32_t slot = base + lane;
        uint32_t x = slot < m ? (uint32_t)D.img[off + slot] : 0u;
        uint32_t c = 0;
        x = run_range16(tab, body + r * p.S, p.S, x, dead, A, &c);
        if (r == p.R - 1 && p.tail) x = run_bytes(tab, body + p.R * p.S, p.tail, x, dead, A, &c);
        if (slot < m) {
          p.slot_end[r * p.cand_stride + slot] = x;
          p.slot_cnt[r * p.cand_stride + slot] = c;
        }
      }
    }

    // 4. main run: each lane runs its merged state over the rest of its row from smem
    uint32_t s = my_sigma, mu = 0;
    const bool run = active && my_conv;
    for (uint32_t blk = 0; blk < nblk && !failed; ++blk) {
      const uint32_t b = blk % kStages;
      const uint32_t bar = smem_u32(sm + bar0 + 8 * b);
      if (!stage_wait(bar, (phase_bits >> b) & 1u, p.wait_budget, p.result)) {
        set_error(p.result, kErrTimeout);
        failed = true;
        break;
      }
      phase_bits ^= 1u << b;
      pending &= ~(1u << b);
      uint4 v[kBox / 16];
      const uint8_t* stg = sm + stage0 + b * kStageBytes + lane * kBox;
#pragma unroll
      for (uint32_t i = 0; i < kBox / 16; ++i)
        v[i] = *reinterpret_cast<const uint4*>(stg + ((i ^ (lane & 7u)) * 16u));
      __syncwarp();
      if (blk + kStages < nblk) {
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_expect_tx(bar, kStageBytes);
          tma_load_2d(smem_u32(sm + stage0 + b * kStageBytes), &tmap, bar,
                      (int32_t)((blk + kStages) * kBox), (int32_t)row0);
        }
        pending |= 1u << b;
      }
      if (run) {
        const uint32_t col0 = blk * kBox;
#pragma unroll
        for (uint32_t i = 0; i < kBox / 16; ++i) {
          if (col0 + i * 16u >= my_t) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              s = tab.next(s, tab.col(byte_of(v[i], q)));
              mu += (s >= A);
            }
          }
        }
      }
    }
    if (failed) continue;
    if (run && myrow == p.R - 1 && p.tail) s = run_bytes(tab, body + p.R * p.S, p.tail, s, dead, A, &mu);
    const uint32_t E = s;  // main end (assumes the row's start reaches my_sigma at my_t)

    // 5. the chunk's end state is known now if every row merged
    const bool fast = __ballot_sync(kFull, active && !my_conv) == 0;
    const bool skip = (int64_t)j == p.skip_publish;
    const uint32_t E_last = __shfl_sync(kFull, E, nrows - 1);
    if (fast && lane == 0 && !skip) st_release(&p.status[j], pack_status(kFlagMapped, 0, E_last, 0));

    // rows k >= 1: start = end of row k-1 (fast path), count the merged prefix [0, t)
    uint32_t x_k = __shfl_up_sync(kFull, E, 1);
    uint32_t cnt_k = 0, dies_k = 0;
    if (fast && active && lane >= 1) {
      if (x_k == dead) {
        dies_k = 1;
      } else {
        uint32_t pre = 0;
        const uint32_t y = run_range16(tab, body + myrow * p.S, my_t, x_k, dead, A, &pre);
        if (y == dead) {
          dies_k = 1;
          cnt_k = pre;
        } else {
          if (y != my_sigma) set_error(p.result, kErrInternal);
          cnt_k = pre + mu;
          dies_k = (E == dead);
        }
      }
    }

    // 6. start state of the chunk: the end state published by chunk j-1
    uint32_t s_j = p.init_state;
    if (j > 0) {
      unsigned long long w = 0;
      if (lane == 0) {
        const long long t0 = clock64();
        for (;;) {
          w = ld_acquire(&p.status[j - 1]);
          if ((w >> 62) != 0) break;
          if ((uint64_t)(clock64() - t0) > p.wait_budget || read_error(p.result)) {
            set_error(p.result, kErrTimeout);
            w = 0;
            break;
          }
        }
      }
      w = __shfl_sync(kFull, w, 0);
      if ((w >> 62) == 0) continue;  // failed: the error word is set
      s_j = (uint32_t)((w >> 45) & 0xFFFFu);
      if (s_j >= D.n) {  // never happens for a consistent status word; keep indices valid
        set_error(p.result, kErrInternal);
        s_j = 0;
      }
    }

    uint32_t E_chunk = E_last;
    if (fast) {
      if (lane == 0) {
        x_k = s_j;
        if (j == 0) {
          cnt_k = head_cnt + mu;
          dies_k = (E == dead);
        } else if (s_j == dead) {
          dies_k = 1;
          cnt_k = 0;
        } else {
          uint32_t pre = 0;
          const uint32_t y = run_range16(tab, body + myrow * p.S, my_t, s_j, dead, A, &pre);
          if (y == dead) {
            dies_k = 1;
            cnt_k = pre;
          } else {
            if (y != my_sigma) set_error(p.result, kErrInternal);
            cnt_k = pre + mu;
            dies_k = (E == dead);
          }
        }
      }
    } else {
      // slow path: walk the rows in order from s_j (lane 0 works, the lanes keep results)
      uint32_t x = s_j;
      for (uint32_t k = 0; k < nrows; ++k) {
        const uint32_t tk = __shfl_sync(kFull, my_t, k);
        const uint32_t sk = __shfl_sync(kFull, my_sigma, k);
        const uint32_t Ek = __shfl_sync(kFull, E, k);
        const uint32_t muk = __shfl_sync(kFull, mu, k);
        const uint32_t ck = __shfl_sync(kFull, my_conv, k);
        const uint32_t hk = __shfl_sync(kFull, head_cnt, k);
        uint32_t cnt = 0, xin = x;
        if (lane == 0) {
          const uint64_t r = row0 + k;
          if (x == dead) {
            cnt = 0;
          } else if (r == 0) {
            cnt = hk + muk;
            x = Ek;
          } else if (ck) {
            uint32_t pre = 0;
            const uint32_t y = run_range16(tab, body + r * p.S, tk, x, dead, A, &pre);
            if (y == dead) {
              cnt = pre;
              x = dead;
            } else {
              if (y != sk) set_error(p.result, kErrInternal);
              cnt = pre + muk;
              x = Ek;
            }
          } else {
            const uint32_t cls =
                p.enum_all ? D.n_classes : (uint32_t)D.byte_class[ldg8(body + r * p.S - 1)];
            const uint32_t slot = D.rank[(uint64_t)cls * D.n + x];
            if (slot == kNoSlot) {
              set_error(p.result, kErrInternal);
              x = 0;  // any valid state: the call reports an error
            } else {
              cnt = p.slot_cnt[r * p.cand_stride + slot];
              x = p.slot_end[r * p.cand_stride + slot];
            }
          }
        }
        xin = __shfl_sync(kFull, xin, 0);
        cnt = __shfl_sync(kFull, cnt, 0);
        x = __shfl_sync(kFull, x, 0);
        if (lane == k) {
          x_k = xin;
          cnt_k = cnt;
          dies_k = (x == dead);
        }
      }
      E_chunk = x;
      if (lane == 0 && !skip) st_release(&p.status[j], pack_status(kFlagMapped, 0, E_chunk, 0));
    }

    // 7. aggregate: counts up to and including the first row whose run dies
    const unsigned dmask = __ballot_sync(kFull, active && dies_k);
    const uint32_t first_dead = dmask ? (uint32_t)(__ffs(dmask) - 1) : 32u;
    uint64_t c = (active && lane <= first_dead) ? cnt_k : 0;
    uint64_t csum = c;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) csum += __shfl_xor_sync(kFull, csum, d);
    const Pfx agg = {dmask ? 1u : 0u, csum};
    if (lane == 0 && !skip)
      st_release(&p.status[j], pack_status(kFlagAggregate, agg.dead, E_chunk, agg.count));

    // 8. decoupled look-back for the exclusive prefix
    Pfx ex = {0, 0};
    if (j > 0) {
      int64_t base = (int64_t)j - 1;
      bool ok = true;
      for (;;) {
        const int64_t idx = base - (int64_t)lane;
        unsigned long long w = 0;
        unsigned inc = 0;
        uint32_t limit = 31;
        const long long t0 = clock64();
        for (;;) {
          w = idx >= 0 ? ld_acquire(&p.status[idx]) : ((unsigned long long)kFlagInclusive << 62);
          const uint32_t flag = (uint32_t)(w >> 62);
          inc = __ballot_sync(kFull, flag == kFlagInclusive);
          const unsigned notready = __ballot_sync(kFull, flag < kFlagAggregate);
          limit = inc ? (uint32_t)(__ffs(inc) - 1) : 31u;
          const unsigned need = limit == 31 ? kFull : ((1u << (limit + 1)) - 1u);
          if (!(notready & need)) break;
          bool stop = false;
          if (lane == 0)
            stop = (uint64_t)(clock64() - t0) > p.wait_budget || read_error(p.result);
          if (__shfl_sync(kFull, stop, 0)) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
        Pfx v = {0, 0};
        if (lane <= limit) {
          v.dead = (uint32_t)((w >> 61) & 1u);
          v.count = w & kCountMask;
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          Pfx o;
          o.dead = __shfl_down_sync(kFull, v.dead, d);
          o.count = __shfl_down_sync(kFull, v.count, d);
          if (lane + d < 32) v = pfx_op(o, v);
        }
        Pfx win;
        win.dead = __shfl_sync(kFull, v.dead, 0);
        win.count = __shfl_sync(kFull, v.count, 0);
        ex = pfx_op(win, ex);
        if (inc) break;
        base -= 32;
      }
      if (!ok) {
        set_error(p.result, kErrTimeout);
        continue;
      }
    }
    const Pfx inc = pfx_op(ex, agg);
    if (lane == 0 && !skip)
      st_release(&p.status[j], pack_status(kFlagInclusive, inc.dead, E_chunk, inc.count));

    // 9. per-row records for the emit pass
    if (p.segrec != nullptr) {
      const bool live_row = active && !ex.dead && lane <= first_dead;
      uint64_t rc = live_row ? cnt_k : 0;
      uint64_t incl = rc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += o;
      }
      if (active) {
        SegRec sr;
        sr.x = live_row ? x_k : dead;
        sr.count = (uint32_t)rc;
        sr.offset = ex.count + incl - rc;
        p.segrec[myrow] = sr;
      }
    }
    if (j == p.n_chunks - 1 && lane == 0) {
      p.result->final_state = inc.dead ? dead : E_chunk;
      p.result->count = inc.count;
    }
  }

  // drain stages still in flight before the CTA may release its shared memory
  for (uint32_t b = 0; b < kStages; ++b) {
    if (pending & (1u << b)) {
      const uint32_t bar = smem_u32(sm + bar0 + 8 * b);
      const long long t0 = clock64();
      while (!mbar_try_wait(bar, (phase_bits >> b) & 1u)) {
        if ((uint64_t)(clock64() - t0) > p.wait_budget) break;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Emit pass: one thread per row with matches, re-run from the resolved start.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
__global__ void __launch_bounds__(256) k_emit(const ScanParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw;
  const DeviceDfa& D = p.dfa;
  {
    const uint4* src = reinterpret_cast<const uint4*>(D.colmap);
    uint4* dst = reinterpret_cast<uint4*>(sm + p.smem_colmap_off);
    for (uint32_t i = threadIdx.x; i < 1024 / 16; i += blockDim.x) dst[i] = src[i];
    if (LAYOUT != kClassGlobal) {
      const uint4* ts = reinterpret_cast<const uint4*>(D.table);
      uint4* td = reinterpret_cast<uint4*>(sm + p.smem_table_off);
      for (uint32_t i = threadIdx.x; i < D.table_bytes / 16; i += blockDim.x) td[i] = ts[i];
    }
  }
  __syncthreads();
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.table_off = p.smem_table_off;
  tab.colmap_off = p.smem_colmap_off;
  tab.gtable = D.table;
  tab.rowbytes = D.rowbytes;
  const uint32_t A = D.first_accept;
  const uint32_t dead = D.dead;
  const uint8_t* body = p.text + p.h;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < p.R;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const SegRec sr = p.segrec[r];
    if (sr.count == 0 || sr.offset >= p.capacity) continue;
    uint64_t o = sr.offset;
    const uint64_t end = (sr.offset + sr.count < p.capacity) ? sr.offset + sr.count : p.capacity;
    uint32_t x = sr.x;
    if (r == 0) {
      for (uint64_t i = 0; i < p.h && o < end; ++i) {
        x = tab.next(x, tab.col(ldg8(p.text + i)));
        if (x >= A) p.positions[o++] = i;
      }
    }
    const uint8_t* rowp = body + r * p.S;
    const uint64_t gbase = p.h + r * p.S;
    for (uint64_t off = 0; off < p.S && o < end; off += 16) {
      const uint4 v = ldg16(rowp + off);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        x = tab.next(x, tab.col(byte_of(v, i)));
        if (x >= A && o < end) p.positions[o++] = gbase + off + (uint64_t)i;
      }
    }
    if (r == p.R - 1) {
      const uint64_t tb = p.h + p.R * p.S;
      for (uint64_t i = 0; i < p.tail && o < end; ++i) {
        x = tab.next(x, tab.col(ldg8(p.text + tb + i)));
        if (x >= A) p.positions[o++] = tb + i;
      }
    }
    (void)dead;
  }
}

// ---------------------------------------------------------------------------------------
// Texts too short for one row: a single thread runs the plain loop on the device.
// ---------------------------------------------------------------------------------------
template <int LAYOUT, int ESIZE>
__global__ void k_tiny(const ScanParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw;
  const DeviceDfa& D = p.dfa;
  {
    const uint4* src = reinterpret_cast<const uint4*>(D.colmap);
    uint4* dst = reinterpret_cast<uint4*>(sm + p.smem_colmap_off);
    for (uint32_t i = threadIdx.x; i < 1024 / 16; i += blockDim.x) dst[i] = src[i];
    if (LAYOUT != kClassGlobal) {
      const uint4* ts = reinterpret_cast<const uint4*>(D.table);
      uint4* td = reinterpret_cast<uint4*>(sm + p.smem_table_off);
      for (uint32_t i = threadIdx.x; i < D.table_bytes / 16; i += blockDim.x) td[i] = ts[i];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  Tab<LAYOUT, ESIZE> tab;
  tab.sm = sm;
  tab.table_off = p.smem_table_off;
  tab.colmap_off = p.smem_colmap_off;
  tab.gtable = D.table;
  tab.rowbytes = D.rowbytes;
  uint32_t x = p.init_state;
  uint64_t cnt = 0;
  for (uint64_t i = 0; i < p.n; ++i) {
    if (x == D.dead) break;
    x = tab.next(x, tab.col(ldg8(p.text + i)));
    if (x >= D.first_accept) {
      if (p.positions && cnt < p.capacity) p.positions[cnt] = i;
      ++cnt;
    }
  }
  p.result->final_state = x;
  p.result->count = cnt;
}

// Launch wrappers, instantiated in the per-layout translation units.
template <int LAYOUT, int ESIZE, int P>
cudaError_t launch_spec_scan(const CUtensorMap& tmap, const ScanParams& p, int grid, int block,
                             size_t smem, cudaStream_t stream) {
  auto kern = k_spec_scan<LAYOUT, ESIZE, P>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, stream>>>(tmap, p);
  return cudaGetLastError();
}

template <int LAYOUT, int ESIZE>
cudaError_t launch_emit(const ScanParams& p, int grid, int block, size_t smem, cudaStream_t stream) {
  auto kern = k_emit<LAYOUT, ESIZE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int LAYOUT, int ESIZE>
cudaError_t launch_tiny(const ScanParams& p, size_t smem, cudaStream_t stream) {
  auto kern = k_tiny<LAYOUT, ESIZE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, 128, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace parem
