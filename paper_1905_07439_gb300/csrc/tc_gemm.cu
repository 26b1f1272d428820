// Leaf products M_rho = S_rho T_rho (Section 2.1.1, F^(0) the standard product) on the
// 5th-generation tensor cores, batched over all R^L leaves, with the decode of
// Eq. recursive-random-formula fused into the epilogue.
//
// Persistent, warp-specialized kernel, one CTA per SM (192 threads; two per SM for small
// plain leaves, see kTwoPerSm):
//   warp 0     one thread issues TMA loads of the S tile (K-major) and the T tile (MN-major:
//              T is stored row-major with n contiguous) with the 128-byte swizzle into a ring
//              of shared-memory stages (mbarrier full/empty handshake);
//   warp 1     allocates TMEM (two fp32 accumulators of 128 x BN; for bf16x6 and f16x3 two
//              buffers of a main and a cross-term accumulator, drained every 256 (bf16x6) or
//              64 (f16x3) elements of K) and one thread issues
//              tcgen05.mma (M = 128, N = BN, K = 16 bf16/f16 or 8 tf32 per instruction),
//              committing stage releases and accumulator-ready signals;
//   warps 2-5  drain an accumulator with tcgen05.ld (one TMEM lane = one tile row per
//              thread) while the MMA fills the other; each 32 x 32 block passes through
//              shared memory so that the global writes cover whole row segments; they scatter
//              the tile into every C block it feeds: C_IJ += (prod_d w^(node_d)_{i_d j_d r_d})
//              * M_tile, by 16-byte vector reductions into the zeroed C (or plain stores when
//              L = 0 / stored M).
// Split-compensated modes keep hi and lo panels of each operand in a stage and issue
// hi*lo' + lo*hi' + hi*hi' per K step into the same accumulator; the bf16x6 mode keeps three
// panels b0, b1, b2 per operand and issues b0*b2' + b2*b0' + b1*b1' + b0*b1' + b1*b0' +
// b0*b0' (smallest terms first); the f16x3 mode keeps two scaled fp16 panels h0, h1 and issues
// h0*h1' + h1*h0' into a cross-term accumulator and h0*h0' into a main one, and its epilogue
// multiplies each entry by the inverse row and column scales.  Tiles are 256 wide whenever the
// padded leaf size allows it (a stage then holds 48 KB per panel set: four stages plain, two
// split), else 128 wide (six stages plain, three split); bf16x6 tiles are 128 wide with two
// stages of 96 KB, f16x3 tiles 128 wide with three stages of 64 KB.
// Every mbarrier wait is bounded (2 s); on expiry the kernel records RBC_ETIMEOUT in the
// workspace status word, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "convert.cuh"
#include "decode_dest.cuh"
#include "ptx.cuh"
#include "tc_gemm.cuh"

namespace rbc {
namespace {

constexpr int BM = 128;
constexpr int kRowBytes = 128;  // one swizzle row: 64 bf16/f16 or 32 tf32 elements of K
constexpr int kThreads = 192;
// Epilogue staging of stored products: one 32 x 32 fp32 block per epilogue warp, rows padded
// to 36 floats (16-byte aligned rows, four-way bank spread).
constexpr int kStageLd = 36;
constexpr size_t kStageBytes = 4 * 32 * kStageLd * sizeof(float);
constexpr uint64_t kWaitNs = 2000000000ull;
// K blocks (64 elements) per accumulator chunk of the f16x3 mode.  Its main products h0*h0' carry
// 22 significant bits, and the tensor cores' truncating accumulation drops low bits of them
// (biased toward zero where the terms share a sign), so its chunks are shorter than bf16x6's.
constexpr int kChunkF16x3 = 1;

struct Params {
  TcInst one;                 // the instance of a single product
  const TcInst* insts;        // grouped launches: device array of ninst instances
  const CUtensorMap* maps;    // grouped launches: tensor maps, (S, T) per instance
  int ninst;
  int64_t total_tiles;
  uint32_t idesc;
  int* status;
  int stall;  // test hook: the producer issues no copies, so the MMA warp's first wait expires
};

// Instance owning global tile `tile`: the last one whose tile_begin <= tile.
template <bool GROUPED>
__device__ __forceinline__ int find_inst(const Params& p, int64_t tile) {
  if constexpr (!GROUPED) {
    return 0;
  } else {
    int lo = 0, hi = p.ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.insts[mid].tile_begin <= tile) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
}

template <int STAGES>
struct Aux {
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  DestList<float> dl[4];
};

__device__ __forceinline__ void raise_abort(volatile int* abort, int* status) {
  *abort = 1;
  if (status) atomicExch(status, (int)RBC_ETIMEOUT);
}

// Tile order within a leaf: groups of p.group_m tile rows, columns swept inside a group, so
// that the CTAs running at the same time share A row panels and B column panels in L2 (a
// plain row-major order re-streams every B panel from DRAM once per tile row when a leaf's
// operands exceed L2).  group_m = 1 is the row-major order.
__device__ __forceinline__ void tile_coords(int64_t tile, const TcInst& p, int64_t* leaf, int* tm, int* tn) {
  const int64_t per_leaf = (int64_t)p.tiles_m * p.tiles_n;
  *leaf = tile / per_leaf;
  const int r = (int)(tile - *leaf * per_leaf);
  const int per_group = p.group_m * p.tiles_n;
  const int g = r / per_group;
  const int first_m = g * p.group_m;
  const int gm = min(p.group_m, p.tiles_m - first_m);
  const int w = r - g * per_group;
  *tm = first_m + w % gm;
  *tn = w / gm;
}

// Plain 128-wide tiles with two stages (about 84 KB of shared memory, 256 TMEM columns) run
// two CTAs per SM: small leaves (a grouped batch's, when the autotuner picks it, and single
// products' of padded size at most 256), whose tiles have few K blocks and a full-tile
// epilogue, then overlap one CTA's epilogue stores with the other's loads and MMAs.  Every
// other configuration needs more than half of the SM's shared memory, so no other CTA of
// this kernel can share an SM with a pair, and TMEM (512 columns) always suffices.
template <int P, int BN, int STAGES>
constexpr bool kTwoPerSm = P == 1 && BN == 128 && STAGES == 2;

// P: stored panels per operand (1 plain, 2 split [hi | lo], 3 bf16x6 [b0 | b1 | b2]).
// SC: f16x3 (P = 2, scaled fp16 panels [h0 | h1], main and cross-term accumulators).
template <int KIND, int P, int BN, int STAGES, bool GROUPED, bool SC>
__global__ void __launch_bounds__(kThreads, kTwoPerSm<P, BN, STAGES> ? 2 : 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ Tables<float> t, const Params p) {
  static_assert(P >= 1 && P <= 3 && (P < 3 || KIND == 0), "three panels are bf16 only");
  static_assert(!SC || (P == 2 && KIND == 0), "f16x3 keeps two fp16 panels");
  constexpr uint32_t A_BYTES = BM * kRowBytes, B_BYTES = BN * kRowBytes;
  constexpr uint32_t STAGE_BYTES = P * (A_BYTES + B_BYTES);
  constexpr int KSTEPS = kRowBytes / 32;  // MMA K steps per stage (32 bytes of K in A rows)
  constexpr int KELEM = KIND == 0 ? 64 : 32;   // K elements per stage
  constexpr int KINSTR = KIND == 0 ? 16 : 8;   // K elements per MMA instruction
  constexpr uint32_t B_ATOM = KELEM * 128;     // one MN atom column of B: KELEM rows x 128 B
  constexpr int B_BOXES = BN / (kRowBytes / (KIND == 0 ? 2 : 4));
  // kind::f16 reads T MN-major (as stored); kind::tf32 takes only K-major operands, so its
  // right operand is stored transposed (T^T, rows n) and loaded like S.
  constexpr bool BMN = KIND == 0;
  // The tensor cores accumulate in fp32 with truncation, whose error grows with the number of
  // accumulations into one sum.  bf16x6 and f16x3 tiles therefore accumulate chunks of KCH K
  // blocks (256 elements of K) in TMEM, each in two accumulators (main term, cross terms), and
  // the epilogue adds the chunks in fp32 registers with round-to-nearest.  Other modes
  // accumulate a whole tile in one accumulator.
  constexpr bool TWO_ACC = P == 3 || SC;
  constexpr int KCH = P == 3 ? 4 : (SC ? kChunkF16x3 : (1 << 30));
  constexpr int ACC_COLS = TWO_ACC ? 2 * BN : BN;  // TMEM columns of one accumulator buffer
  static_assert(2 * ACC_COLS <= 512, "two accumulator buffers fit TMEM");

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Aux<STAGES>* aux = reinterpret_cast<Aux<STAGES>*>(smem + STAGES * STAGE_BYTES);
  float* ostage = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + ((sizeof(Aux<STAGES>) + 15) & ~(size_t)15));
  volatile int* abort = &aux->abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&aux->full[s], 1);
      ptx::mbar_init(&aux->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&aux->tfull[b], 1);
      ptx::mbar_init(&aux->tempty[b], 4);
    }
    ptx::mbar_init(&aux->drain, 1);
    aux->abort = 0;
    ptx::fence_mbar_init();
    if (!GROUPED) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(&tmB);
    }
  }
  if (warp == 1) {
    ptx::tmem_alloc(&aux->tmem_base, 2 * ACC_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = aux->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t armed = 0, last_par = 0;  // per-stage bit masks for the teardown drain
      int fenced = -1;                   // grouped: instance whose maps were last fenced
      for (int64_t tile = blockIdx.x; tile < p.total_tiles && !*abort && !p.stall; tile += gridDim.x) {
        const int ii = find_inst<GROUPED>(p, tile);
        const TcInst d = GROUPED ? p.insts[ii] : p.one;
        const void* mA = GROUPED ? (const void*)&p.maps[2 * ii] : (const void*)&tmA;
        const void* mB = GROUPED ? (const void*)&p.maps[2 * ii + 1] : (const void*)&tmB;
        if (GROUPED && ii != fenced) {
          ptx::fence_tmap_acquire(mA);
          ptx::fence_tmap_acquire(mB);
          fenced = ii;
        }
        int64_t leaf;
        int tm, tn;
        tile_coords(tile - d.tile_begin, d, &leaf, &tm, &tn);
        const int32_t rowA = (int32_t)(leaf * d.mp + (int64_t)tm * BM);
        const int32_t colB = tn * BN;
        for (int kb = 0; kb < d.nk; ++kb) {
          if (!ptx::wait_bounded(&aux->empty[s], ph ^ 1u, abort, kWaitNs)) {
            raise_abort(abort, p.status);
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          ptx::mbar_arrive_expect_tx(&aux->full[s], STAGE_BYTES);
          const int32_t kx = kb * KELEM;
#pragma unroll
          for (int q = 0; q < P; ++q) ptx::tma_load_2d(st + q * A_BYTES, mA, &aux->full[s], kx + q * d.kpanel, rowA);
          if constexpr (BMN) {
            const int32_t rowB = (int32_t)(leaf * d.mp) + kx;
            constexpr int NBOX = kRowBytes / (KIND == 0 ? 2 : 4);
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
              for (int j = 0; j < B_BOXES; ++j)
                ptx::tma_load_2d(st + P * A_BYTES + q * B_BYTES + j * B_ATOM, mB, &aux->full[s],
                                 colB + j * NBOX + q * d.kpanel, rowB);
          } else {
            const int32_t rowB = (int32_t)(leaf * d.mp) + colB;
#pragma unroll
            for (int q = 0; q < P; ++q)
              ptx::tma_load_2d(st + P * A_BYTES + q * B_BYTES, mB, &aux->full[s], kx + q * d.kpanel, rowB);
          }
          armed |= 1u << s;
          last_par = (last_par & ~(1u << s)) | (ph << s);
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // Wait for every copy this thread started (bounded) before the CTA can exit.
      for (int q = 0; q < STAGES; ++q)
        if (armed & (1u << q)) {
          volatile int never = 0;
          ptx::wait_bounded(&aux->full[q], (last_par >> q) & 1u, &never, kWaitNs);
        }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int s = 0, buf = 0;
      uint32_t ph = 0, aph = 0;
      for (int64_t tile = blockIdx.x; tile < p.total_tiles && !*abort; tile += gridDim.x) {
        const int nk = GROUPED ? p.insts[find_inst<GROUPED>(p, tile)].nk : p.one.nk;
        bool ok = true;
        uint32_t d_tmem = 0;
        for (int kb = 0; kb < nk; ++kb) {
          const int kc = kb % KCH;  // K block inside the current accumulator chunk
          if (kc == 0) {            // a chunk starts: wait for a drained accumulator
            if (!ptx::wait_bounded(&aux->tempty[buf], aph ^ 1u, abort, kWaitNs)) {
              raise_abort(abort, p.status);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            d_tmem = tmem_base + (uint32_t)(buf * ACC_COLS);
          }
          if (!ptx::wait_bounded(&aux->full[s], ph, abort, kWaitNs)) {
            raise_abort(abort, p.status);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t a0 = ptx::smem_u32(smem + s * STAGE_BYTES);
          const uint32_t b0 = a0 + P * A_BYTES;
#pragma unroll
          for (int k = 0; k < KSTEPS; ++k) {
            // descriptors of panel q of A and B at this K step
            uint64_t ad[P], bd[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
              ad[q] = ptx::desc_sw128(a0 + q * A_BYTES + k * 32);
              bd[q] = BMN ? ptx::desc_sw128_mn(b0 + q * B_BYTES + k * KINSTR * 128, 1024, B_ATOM)
                          : ptx::desc_sw128(b0 + q * B_BYTES + k * 32);
            }
            const uint32_t acc = (kc > 0 || k > 0) ? 1u : 0u;
            if constexpr (P == 3) {
              // five cross terms (at most 2^-8 of the leading one) into their own accumulator,
              // b0*b0' alone into the main one: only one truncating accumulation of the main
              // sum per K step
              const uint32_t d_small = d_tmem + (uint32_t)BN;
              ptx::mma<KIND>(d_small, ad[0], bd[2], p.idesc, acc);
              ptx::mma<KIND>(d_small, ad[2], bd[0], p.idesc, 1u);
              ptx::mma<KIND>(d_small, ad[1], bd[1], p.idesc, 1u);
              ptx::mma<KIND>(d_small, ad[0], bd[1], p.idesc, 1u);
              ptx::mma<KIND>(d_small, ad[1], bd[0], p.idesc, 1u);
              ptx::mma<KIND>(d_tmem, ad[0], bd[0], p.idesc, acc);
            } else if constexpr (SC) {
              // h0*h1' + h1*h0' (at most 2^-10 of the leading term) into the cross-term
              // accumulator, h0*h0' alone into the main one
              const uint32_t d_small = d_tmem + (uint32_t)BN;
              ptx::mma<KIND>(d_small, ad[0], bd[1], p.idesc, acc);
              ptx::mma<KIND>(d_small, ad[1], bd[0], p.idesc, 1u);
              ptx::mma<KIND>(d_tmem, ad[0], bd[0], p.idesc, acc);
            } else if constexpr (P == 2) {
              ptx::mma<KIND>(d_tmem, ad[0], bd[1], p.idesc, acc);
              ptx::mma<KIND>(d_tmem, ad[1], bd[0], p.idesc, 1u);
              ptx::mma<KIND>(d_tmem, ad[0], bd[0], p.idesc, 1u);
            } else {
              ptx::mma<KIND>(d_tmem, ad[0], bd[0], p.idesc, acc);
            }
          }
          ptx::mma_commit(&aux->empty[s]);  // stage free once these MMAs have read it
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
          if (kc == KCH - 1 || kb == nk - 1) {
            ptx::mma_commit(&aux->tfull[buf]);  // chunk (or tile) accumulated
            if (++buf == 2) {
              buf = 0;
              aph ^= 1u;
            }
          }
        }
        if (!ok) break;
      }
      // All MMAs issued by this thread complete before TMEM is released.
      ptx::mma_commit(&aux->drain);
      volatile int never = 0;
      ptx::wait_bounded(&aux->drain, 0u, &never, kWaitNs);
    }
  } else {
    // ---------------- epilogue: warps 2..5 ----------------
    const int quarter = warp & 3;  // TMEM lanes this warp may access
    DestList<float>& dl = aux->dl[warp - 2];
    int buf = 0;
    uint32_t aph = 0;
    for (int64_t tile = blockIdx.x; tile < p.total_tiles; tile += gridDim.x) {
      const TcInst d = GROUPED ? p.insts[find_inst<GROUPED>(p, tile)] : p.one;
      int64_t leaf;
      int tm, tn;
      tile_coords(tile - d.tile_begin, d, &leaf, &tm, &tn);
      __syncwarp();  // every lane is done with the previous tile's list
      if (d.epi == 0 && lane == 0) build_dest_list(t, leaf, dl);
      // Output of one 32-column block v of this warp's 32 rows.  Every output goes through
      // shared memory, so that each store (or reduction) instruction covers four whole
      // 128-byte row segments: a lane holds one row of the accumulator, and the 32 x 32 block
      // is re-read by rows.
      auto out_block = [&](const float (&v)[32], int c0) {
        const int64_t col0 = (int64_t)tn * BN + c0;
        float* sb = ostage + (warp - 2) * 32 * kStageLd;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(sb + lane * kStageLd + 4 * q) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        const int64_t row0 = (int64_t)tm * BM + quarter * 32;
        const int cl = (lane & 7) * 4;  // this lane's four columns of the chunk
        if (d.epi == 2) {  // the product, into M (whole padded tiles)
          float* dstb = d.M + leaf * d.strideM + row0 * d.ldm + col0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int r = j * 4 + (lane >> 3);
            *reinterpret_cast<float4*>(dstb + r * d.ldm + cl) = *reinterpret_cast<const float4*>(sb + r * kStageLd + cl);
          }
        } else if (d.epi == 1) {  // L = 0: the product is C (valid rows and columns only)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int r = j * 4 + (lane >> 3);
            const int64_t gr = row0 + r, gc = col0 + cl;
            if (gr >= d.m) continue;
            const float4 x = *reinterpret_cast<const float4*>(sb + r * kStageLd + cl);
            float* dst = d.C + gr * d.ldc + gc;
            if (d.vec_ok && gc + 3 < d.m) {
              *reinterpret_cast<float4*>(dst) = x;
            } else {
              const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (gc + e < d.m) dst[e] = xs[e];
            }
          }
        } else {  // fused decode: coef * product added into every C block the leaf feeds
          for (int di = 0; di < dl.total; ++di) {
            int64_t I, J;
            const float coef = dest_at(dl, di, t.n0, t.L, &I, &J);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int r = j * 4 + (lane >> 3);
              const int64_t gr = row0 + r, gc = col0 + cl;
              if (gr >= d.m) continue;
              const float4 x = *reinterpret_cast<const float4*>(sb + r * kStageLd + cl);
              float* dst = d.C + (I * d.m + gr) * d.ldc + J * d.m + gc;
              if (d.vec_ok && gc + 3 < d.m) {
                ptx::red_add_v4(dst, coef * x.x, coef * x.y, coef * x.z, coef * x.w);
              } else {
                const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (gc + e < d.m) atomicAdd(dst + e, coef * xs[e]);
              }
            }
          }
        }
        __syncwarp();  // the block is read before the next one overwrites it
      };
      int ok = 1;
      if constexpr (TWO_ACC) {
        // chunks of the tile's K: sum main and cross-term accumulators in registers (fp32,
        // round to nearest), releasing each accumulator buffer as soon as it is read
        const int nch = (d.nk + KCH - 1) / KCH;
        float sum[BN];
#pragma unroll
        for (int i = 0; i < BN; ++i) sum[i] = 0.f;
        for (int c = 0; c < nch; ++c) {
          if (lane == 0) ok = ptx::wait_bounded(&aux->tfull[buf], aph, abort, kWaitNs) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) break;
          __syncwarp();
          ptx::tc_fence_after();
          const uint32_t tb = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * ACC_COLS);
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 32) {
            float x[32];
            ptx::tmem_ld32(tb + (uint32_t)(BN + c0), x);  // cross terms
            // f16x3: the low pieces were stored times 2^11 (exact scaling back)
            constexpr float cs = SC ? 1.f / kF16LoScale : 1.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) sum[c0 + i] += SC ? x[i] * cs : x[i];
            ptx::tmem_ld32(tb + (uint32_t)c0, x);         // main term
#pragma unroll
            for (int i = 0; i < 32; ++i) sum[c0 + i] += x[i];
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&aux->tempty[buf]);
          if (++buf == 2) {
            buf = 0;
            aph ^= 1u;
          }
        }
        if (!ok) {
          if (lane == 0) raise_abort(abort, p.status);
          break;
        }
        float rs = 1.f;
        if constexpr (SC) rs = d.rinv[(int64_t)tm * BM + quarter * 32 + lane];  // this lane's row
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float v[32];
          if constexpr (SC) {
            const float4* cs = reinterpret_cast<const float4*>(d.cinv + (int64_t)tn * BN + c0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 c = cs[q];  // powers of two: the products below are exact
              v[4 * q] = sum[c0 + 4 * q] * (rs * c.x);
              v[4 * q + 1] = sum[c0 + 4 * q + 1] * (rs * c.y);
              v[4 * q + 2] = sum[c0 + 4 * q + 2] * (rs * c.z);
              v[4 * q + 3] = sum[c0 + 4 * q + 3] * (rs * c.w);
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = sum[c0 + i];
          }
          out_block(v, c0);
        }
      } else {
        if (lane == 0) ok = ptx::wait_bounded(&aux->tfull[buf], aph, abort, kWaitNs) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) raise_abort(abort, p.status);
          break;
        }
        __syncwarp();
        ptx::tc_fence_after();
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN);
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float v[32];
          ptx::tmem_ld32(tbase + (uint32_t)c0, v);
          if (c0 + 32 == BN) {
            // accumulator fully read: hand it back to the MMA warp before the global writes
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&aux->tempty[buf]);
          }
          out_block(v, c0);
        }
        if (++buf == 2) {
          buf = 0;
          aph ^= 1u;
        }
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, 2 * ACC_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

// 2D map over rows x K elements (row-major, K contiguous) with a box of box_rows x 128 bytes.
bool make_map(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int es, int64_t K, int64_t rows,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(K * es)};
  cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND, int P, int BN, int STAGES, bool GROUPED, bool SC = false>
cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, const Tables<float>& t, const Params& p,
                   cudaStream_t st) {
  constexpr size_t smem =
      (size_t)STAGES * P * (BM + BN) * kRowBytes + ((sizeof(Aux<STAGES>) + 15) & ~(size_t)15) + kStageBytes + 1024;
  static_assert(smem <= 232448, "shared memory budget");
  static_assert(!kTwoPerSm<P, BN, STAGES> || 2 * (smem + 1024) <= 233472, "two CTAs per SM");
  // a CTA of any other configuration takes more than half of the SM's shared memory, so it never
  // shares an SM (and its TMEM) with another CTA of this kernel
  static_assert(kTwoPerSm<P, BN, STAGES> || 2 * (smem + 1024) > 233472, "one CTA per SM");
  auto kern = tc_gemm_kernel<KIND, P, BN, STAGES, GROUPED, SC>;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  // Once per device (never inside a later stream capture): allow the large shared memory.
  static std::mutex mu;
  static bool attr_set[64] = {};
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
      const cudaError_t attr_err =
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (attr_err != cudaSuccess) return attr_err;
      attr_set[dev] = true;
    }
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (kTwoPerSm<P, BN, STAGES> ? 2 : 1) * (int64_t)sms;
  const int64_t grid = p.total_tiles < cap ? p.total_tiles : cap;
  if (grid <= 0) return cudaSuccess;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(ma, mb, t, p);
  return cudaGetLastError();
}

// Kernel variant for a leaf mode, tile width and CTAs per SM (2: plain 128-wide tiles only).
template <bool GROUPED>
cudaError_t dispatch(int leaf, int bn, int ctas, const CUtensorMap& ma, const CUtensorMap& mb,
                     const Tables<float>& t, const Params& p, cudaStream_t st) {
  const bool tf32 = leaf == RBC_LEAF_TF32 || leaf == RBC_LEAF_3XTF32;
  const bool split = leaf == RBC_LEAF_3XTF32 || leaf == RBC_LEAF_3XBF16;
  if (leaf == RBC_LEAF_BF16X6) {
    // three 16 KB panels of A and of B per stage: two stages of 96 KB at 128-wide tiles
    if (ctas != 1 || bn != 128) return cudaErrorInvalidValue;
    return launch<0, 3, 128, 2, GROUPED>(ma, mb, t, p, st);
  }
  if (leaf == RBC_LEAF_F16X3) {
    // two 16 KB panels of A and of B per stage: three stages of 64 KB at 128-wide tiles (two
    // accumulator buffers of main and cross terms fill TMEM)
    if (ctas != 1 || bn != 128) return cudaErrorInvalidValue;
    return launch<0, 2, 128, 3, GROUPED, true>(ma, mb, t, p, st);
  }
  if (ctas != 1) {
    if (ctas != 2 || split || bn != 128) return cudaErrorInvalidValue;
    return tf32 ? launch<1, 1, 128, 2, GROUPED>(ma, mb, t, p, st) : launch<0, 1, 128, 2, GROUPED>(ma, mb, t, p, st);
  }
  // split tiles of width 256 hold two panel pairs per stage (96 KB): two stages fit
  if (tf32) {
    if (split) {
      if (bn == 256) return launch<1, 2, 256, 2, GROUPED>(ma, mb, t, p, st);
      return launch<1, 2, 128, 3, GROUPED>(ma, mb, t, p, st);
    }
    if (bn == 256) return launch<1, 1, 256, 4, GROUPED>(ma, mb, t, p, st);
    return launch<1, 1, 128, 6, GROUPED>(ma, mb, t, p, st);
  }
  if (split) {
    if (bn == 256) return launch<0, 2, 256, 2, GROUPED>(ma, mb, t, p, st);
    return launch<0, 2, 128, 3, GROUPED>(ma, mb, t, p, st);
  }
  if (bn == 256) return launch<0, 1, 256, 4, GROUPED>(ma, mb, t, p, st);
  return launch<0, 1, 128, 6, GROUPED>(ma, mb, t, p, st);
}

uint32_t leaf_idesc(int leaf, int bn) {
  const bool tf32 = leaf == RBC_LEAF_TF32 || leaf == RBC_LEAF_3XTF32;
  const uint32_t fmt = tf32 ? 2u : ((leaf == RBC_LEAF_F16 || leaf == RBC_LEAF_F16X3) ? 0u : 1u);
  return ptx::idesc(fmt, fmt, BM, bn, tf32 ? 0u : 1u);
}

}  // namespace

int64_t tc_pad(int64_t m) { return (m + 127) / 128 * 128; }

int tc_default_bn(int leaf, int64_t mp) {
  if (leaf == RBC_LEAF_BF16X6) return 128;  // a 256-wide stage of three panel pairs does not fit twice
  if (leaf == RBC_LEAF_F16X3) return 128;   // two accumulator buffers of main and cross terms: 4 x 128 columns
  return mp % 256 == 0 ? 256 : 128;
}

int tc_default_group(int leaf, int64_t mp, int64_t K) {
  const bool tf32 = leaf == RBC_LEAF_TF32 || leaf == RBC_LEAF_3XTF32;
  const double leaf_bytes = 2.0 * (double)mp * (double)K * (tf32 ? 4 : 2);
  // group tile rows only when one leaf's operands do not fit in L2 (about 64 MB per die)
  return leaf_bytes > 64.0 * (1 << 20) ? 8 : 1;
}

bool tc_prepare_instance(const TcGemmArgs& a, int bn, int group_m, int64_t tile_begin, TcInst* d, void* maps2) {
  const bool tf32 = a.leaf == RBC_LEAF_TF32 || a.leaf == RBC_LEAF_3XTF32;
  const int es = tf32 ? 4 : 2;
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : ((a.leaf == RBC_LEAF_F16 || a.leaf == RBC_LEAF_F16X3) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  if (a.mp % 128 || a.mp % bn) return false;
  if (a.leaf == RBC_LEAF_F16X3 && (!a.rinv || !a.cinv)) return false;
  const int64_t rows = a.leaves * a.mp;
  if (rows > INT32_MAX || a.K > INT32_MAX) return false;
  CUtensorMap* m = static_cast<CUtensorMap*>(maps2);
  // A: rows of S (K contiguous), boxes 128 rows x 128 B.  B: T^T rows (tf32) like A, or T rows
  // (k, n contiguous) in boxes of (K elements per stage) rows x 128 B of n.
  if (!make_map(&m[0], a.S, dt, es, a.K, rows, BM) ||
      !make_map(&m[1], a.T, dt, es, a.K, rows, tf32 ? bn : kRowBytes / es))
    return false;
  TcInst x{};
  x.m = a.m;
  x.mp = a.mp;
  x.leaves = a.leaves;
  x.tile_begin = tile_begin;
  x.tiles_m = (int)(a.mp / BM);
  x.tiles_n = (int)(a.mp / bn);
  x.group_m = group_m;
  x.nk = (int)(a.mp / (kRowBytes / es));
  x.kpanel = (int)a.mp;
  x.epi = a.store_m ? 2 : (a.direct ? 1 : 0);
  x.vec_ok = ((uintptr_t)a.C % 16 == 0) && a.ldc % 4 == 0 && a.m % 4 == 0;
  x.C = static_cast<float*>(a.C);
  x.ldc = a.ldc;
  x.M = static_cast<float*>(a.M);
  x.ldm = a.mp;
  x.strideM = a.strideM;
  x.rinv = a.rinv;
  x.cinv = a.cinv;
  *d = x;
  return true;
}

int64_t tc_instance_tiles(const TcInst& d) { return d.leaves * d.tiles_m * d.tiles_n; }

cudaError_t launch_tc_gemm(const Tables<float>& t, const TcGemmArgs& a, cudaStream_t st) {
  // Small plain leaves (padded size at most 256) run 128-wide tiles, two CTAs per SM: their
  // tiles have at most four K blocks, and the second CTA overlaps one CTA's epilogue with the
  // other's loads (bf16 Laderman leaves of 243 -> 256: 1.05 -> 0.92 ms per launch; at 512 the
  // 256-wide single CTA per SM stays faster, 0.76 against 0.93 ms).
  const bool pair = !(a.leaf == RBC_LEAF_3XBF16 || a.leaf == RBC_LEAF_3XTF32 || a.leaf == RBC_LEAF_BF16X6 ||
                      a.leaf == RBC_LEAF_F16X3) &&
                    a.mp <= 256;
  const int bn = pair ? 128 : tc_default_bn(a.leaf, a.mp);
  CUtensorMap maps[2];
  Params p{};
  if (!tc_prepare_instance(a, bn, tc_default_group(a.leaf, a.mp, a.K), 0, &p.one, maps))
    return cudaErrorInvalidValue;
  p.total_tiles = tc_instance_tiles(p.one);
  p.idesc = leaf_idesc(a.leaf, bn);
  p.status = a.status;
  p.stall = a.stall;
  return dispatch<false>(a.leaf, bn, pair ? 2 : 1, maps[0], maps[1], t, p, st);
}

cudaError_t launch_tc_gemm_grouped(const TcGroupArgs& g, cudaStream_t st) {
  static const Tables<float> kNoTables{};  // grouped launches store the leaf products (no fused decode)
  Params p{};
  p.insts = g.insts;
  p.maps = static_cast<const CUtensorMap*>(g.maps);
  p.ninst = g.ninst;
  p.total_tiles = g.total_tiles;
  p.idesc = leaf_idesc(g.leaf, g.bn);
  p.status = g.status;
  CUtensorMap unused{};
  return dispatch<true>(g.leaf, g.bn, g.ctas, unused, unused, kNoTables, p, st);
}

}  // namespace rbc
