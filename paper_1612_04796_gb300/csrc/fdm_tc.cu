// Fast diagonalisation of the subdomain problems on the tensor cores
// (Section 3.1), FP32 multigrid path: tcgen05.mma with TF32 inputs and FP32
// accumulation in tensor memory.
//
// Each of the six 1D passes of
//   du_s = (Sz(x)Sy(x)Sx) (Lx (+) Ly (+) Lz)^{-1} (Sz^T(x)Sy^T(x)Sx^T) r_s
// (x, y, z forward; z, y, x backward with the weights folded into SW)
// contracts every 1D line of the tiles of a group of G subdomains with one
// m x m factor:
//   forward   out[line][p] = sum_a in[line][a] S[a][p]
//   backward  out[line][a] = sum_p in[line][p] SW[a][p]
//
// Layout.  The lines of a pass are numbered so that the index that becomes
// the contraction index K of the NEXT pass runs fastest, padded to a multiple
// of four, and Q = 4 (or, for tiles whose pass output would not fit the 512
// tensor-memory columns that way, Q = 2) consecutive lines form one row of
// the MMA operand A (a "quad" or "pair": its lines side by side along K, line
// i at K offset i K_a, K_a = m rounded up to 4).  A sits in shared memory in
// the no-swizzle K-major canonical layout (8-row x 16-byte core matrices,
// K-adjacent core matrices LBO bytes apart, 8-row groups SBO = Q K_a / 4 LBO
// bytes apart).  Per 128-row tile and line i of the row one MMA (M = 128,
// N = N_pad, K = 8 per step, K_pad = m rounded up to 8 in all) writes the
// outputs of that line to tensor-memory columns (Q t + i) N_pad .. (the last
// tile is anchored at the end of the rows, overlapping its predecessor, whose
// rows it does not write back, so no padding tile is stored); one thread
// issues them and waits on the commit mbarrier while the others sleep in a
// block barrier.  Where K_a < K_pad the MMA of line i reads the first K
// positions of line i + 1 (or, past the last row group, one spare core
// matrix) against zero rows of B.  Every warp then reads its 32 lanes (rows)
// back with tcgen05.ld: a thread holds, for each output index o, the Q values
// of its row's lines -- Q consecutive K of the next pass -- and stores them
// with one 16-byte (Q = 4) or 8-byte (Q = 2) store into the next layout, in
// place (the whole pass output is held in tensor memory).  The division by lam_x + lam_y + lam_z is applied
// between the two z passes (whose lines are the same), and the last pass
// writes the weighted correction tile to global memory in the layout of the
// CUDA-core kernels.
//
// Padding: K is padded to a multiple of 8 and N to a multiple of 16 with zero
// rows / columns in B, so padded K positions of A (which hold finite values:
// A starts zeroed and only data is stored) add nothing; padding lines carry
// finite garbage into padded K positions only.  Values are rounded to TF32
// (to nearest) when stored as MMA inputs.  Every wait is bounded in time; on a
// timeout the kernel sets the status word, leaves its loops and still frees
// its tensor memory (mg_selftest_bounded_wait runs the kernel with a barrier
// that nothing arrives on to check exactly that).
#include <stdint.h>

#include <algorithm>

#include "mg_internal.h"

namespace mgdg {
namespace {

// Threads per CTA: 256 where several CTAs share an SM, 512 where one CTA has
// the SM (the largest tiles: the write-backs and the gather are bound by the
// issue rate of the CTA's warps).  Warp w reads tensor-memory lanes 32 (w % 4) ..
constexpr int kTcThreads = 256;
constexpr int kTcThreadsWide = 512;
constexpr int kTcRows = 128;     // MMA tile height M (quads)
constexpr long long kTcWaitCycles = 4000000000LL;  // about 2 s at the maximum SM clock
constexpr long long kTcSelfTestWaitCycles = 20000000LL;  // about 10 ms
constexpr int kPassDir[6] = {0, 1, 2, 2, 1, 0};

struct TcPass {
  int dir;        // direction contracted
  int lines;      // lines per subdomain (multiple of 4)
  int fast;       // padded extent of the fastest line index
  int ka;         // K stride of a line in A: m rounded up to 4
  int kp;         // K of the MMAs: m rounded up to 8
  int np;         // N padded to a multiple of 16
  int quads;      // rows of A: G * lines / Q
  int tiles;      // 128-row tiles
  int last0;      // first row of the last tile: anchored at the end of the rows (rounded up
                  // to 8) when there are several tiles, so the buffer needs no padding tile
  uint32_t boff;  // byte offset of this pass's factor in the B region
};

struct TcArgs {
  const float* tab;
  const float* r;
  float* corr;
  int* status;
  int64_t Ne;
  int nx, ny, nz, n;
  int md[3], mp[3], nod[3];  // widths, widths rounded up to 4, layers
  int G;                     // subdomains per group
  int q;                     // lines per row of A (4 or 2)
  int64_t S[3], SW[3], dinvp;
  TcPass pass[6];
  uint32_t a_bytes;    // bytes of the quad buffer A; the factor region B follows
  int lbo_a;           // bytes between K-adjacent core matrices of A (144: bank spread, or 128)
  int b_resident;      // 1: all six factors loaded once; 0: reloaded per pass at offset 0
  uint32_t tmem_cols;  // power of two >= 32
  long long wait_cycles;  // limit of each mbarrier wait
  int self_test;          // 1: issue no MMA and no commit, so the first wait runs out
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major, M = 128.
__device__ __forceinline__ uint32_t tc_idesc(int np) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Wait for completion `phase` of the mbarrier, bounded in time.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase, long long limit) {
  const long long t0 = clock64();
  uint32_t done = 0;
  while (true) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase));
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// FP32 -> TF32, round to nearest (ties away), kept in an FP32 container.
__device__ __forceinline__ float tc_tf32(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

__device__ __forceinline__ float4 tc_tf32x4(float a, float b, float c, float d) {
  return make_float4(tc_tf32(a), tc_tf32(b), tc_tf32(c), tc_tf32(d));
}

// Float index of K position kk (a multiple of Q for the vector stores) of
// line `line` (group-wide numbering) in the layout of Q lines per row, line
// stride ka along K.
template <int Q>
__device__ __forceinline__ int tc_at(int line, int kk, int ka, int lbo_w) {
  const int q = line / Q, k = (line % Q) * ka + kk;
  return (q & 7) * 4 + (q >> 3) * (Q * ka / 4 * lbo_w) + (k & 3) + (k >> 2) * lbo_w;
}

// Float index of (n, k) in the layout of B (LBO 128, SBO 32 kp bytes).
__device__ __forceinline__ int tc_at_b(int nn, int k, int kp) {
  return (nn & 7) * 4 + (nn >> 3) * 8 * kp + (k & 3) + (k >> 2) * 32;
}

__device__ __forceinline__ void tc_sub_node(int a, int n, int no, int* de, int* ii) {
  if (a < no) { *de = -1; *ii = n - no + a; }
  else if (a < no + n) { *de = 0; *ii = a - no; }
  else { *de = 1; *ii = a - no - n; }
}

__device__ __forceinline__ int tc_wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// The 1D factor of pass p: B[n][k] = S[k][n] (forward) or SW[n][k] (backward), zero padded.
template <int NT>
__device__ __forceinline__ void tc_load_factor(const TcArgs& a, int p, float* Bp, int tid) {
  const TcPass& ps = a.pass[p];
  const int d = ps.dir, m = a.md[d];
  const float* __restrict__ F = a.tab + (p < 3 ? a.S[d] : a.SW[d]);
  for (int i = tid; i < ps.np * ps.kp; i += NT) {
    const int nn = i / ps.kp, k = i - nn * ps.kp;
    float v = 0.f;
    if (nn < m && k < m) v = tc_tf32((p < 3) ? F[k * m + nn] : F[nn * m + k]);
    Bp[tc_at_b(nn, k, ps.kp)] = v;
  }
}

// Read pass P's output back and store it where the next pass (or the
// correction) needs it.  The row of a thread holds lines f0 .. f0 + Q - 1
// (fast index) of slow index sl of subdomain g; their output o goes to
// next-pass line nl(o) at K = f0 .. f0 + Q - 1 (P = 0, 1, 3, 4), to the same
// lines at K = o (P = 2, times the inverse eigenvalue sums), or to the
// correction (P = 5).
template <int Q>
__device__ __forceinline__ void tc_store_row(float* dst, const float (&v)[Q][16], int j) {
  if constexpr (Q == 4) {
    *reinterpret_cast<float4*>(dst) = tc_tf32x4(v[0][j], v[1][j], v[2][j], v[3][j]);
  } else {
    *reinterpret_cast<float2*>(dst) = make_float2(tc_tf32(v[0][j]), tc_tf32(v[1][j]));
  }
}

template <int P, int Q, int NT>
__device__ __forceinline__ void tc_writeback(const TcArgs& a, float* A, uint32_t tmem, int warp, int lane, int64_t s0,
                                             bool ok) {
  const TcPass& ps = a.pass[P];
  const int mx = a.md[0], my = a.md[1], mz = a.md[2];
  const int m = a.md[ps.dir];
  const int lbo_w = a.lbo_a / 4;
  const int kan = P < 5 ? a.pass[P + 1].ka : 0;
  const int Ln = P < 5 ? a.pass[P + 1].lines : 0;
  const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
  // work items (tile, 16-column chunk), shared out over the NT / 128 groups of
  // four warps (one warp per 32-lane quarter of the tile)
  const int nch = ps.np / 16;
  int t = -1, g = 0, l0 = 0, f0 = 0, sl = 0;
  bool valid = false;
  for (int it = warp >> 2; it < ps.tiles * nch; it += NT / 128) {
    const int tt = it / nch, c0 = (it - tt * nch) * 16;
    if (tt != t) {
      t = tt;
      const int t0 = t == ps.tiles - 1 ? ps.last0 : t * kTcRows;  // rows below t * 128 belong to earlier tiles
      const int quad = t0 + (warp & 3) * 32 + lane;
      const int line0 = Q * quad;
      g = line0 / ps.lines;
      l0 = line0 - g * ps.lines;
      f0 = l0 % ps.fast;
      sl = l0 / ps.fast;
      valid = ok && quad < ps.quads && quad >= t * kTcRows && s0 + g < a.Ne;
    }
    {
      float v[Q][16];
#pragma unroll
      for (int i = 0; i < Q; ++i) tc_ld16(tmem + lanes + (uint32_t)((Q * t + i) * ps.np + c0), v[i]);
      tc_ld_wait();
      if (!valid) continue;
      if (P == 2) {
        // same lines, K = o: four consecutive o per 16-byte store, times 1 / (lam_x + lam_y + lam_z)
        const float* __restrict__ dv = a.tab + a.dinvp + (int64_t)(f0 + a.mp[1] * sl) * a.mp[2] + c0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            if (c0 + j < m) {
              const float4 w = __ldg(reinterpret_cast<const float4*>(dv + i * a.mp[2] + j));
              *reinterpret_cast<float4*>(A + tc_at<Q>(g * Ln + l0 + i, c0 + j, kan, lbo_w)) =
                  tc_tf32x4(v[i][j] * w.x, v[i][j + 1] * w.y, v[i][j + 2] * w.z, v[i][j + 3] * w.w);
            }
          }
        }
      } else if (P == 5) {
        // lines (b, c), o = a: the correction tile, node a + mx (b + my c)
        float* __restrict__ out = a.corr + (s0 + g) * ((int64_t)mx * my * mz) + mx * (f0 + my * sl) + c0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (f0 + i < my) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < m) out[i * mx + j] = v[i][j];
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int o = c0 + j;
          if (o < m) {
            int nl;
            if (P == 0) nl = sl + a.mp[2] * o;       // (b, c) -> (c, px = o), K = b
            else if (P == 1) nl = o + a.mp[1] * sl;  // (c, px) -> (q = o, px), K = c
            else if (P == 3) nl = sl + a.mp[0] * o;  // (q, px) -> (px, c = o), K = q
            else nl = o + a.mp[1] * sl;              // (px, c) -> (b = o, c), K = px
            tc_store_row<Q>(A + tc_at<Q>(g * Ln + nl, f0, kan, lbo_w), v, j);
          }
        }
      }
    }
  }
}

template <int Q, int NT>
__global__ void __launch_bounds__(NT) k_fdm_tc(TcArgs a) {
  pdl_entry();
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ uint32_t pending_phase;  // phase of the commit a timed-out wait was waiting for
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* A = reinterpret_cast<float*>(tc_smem);
  float* B = reinterpret_cast<float*>(tc_smem + a.a_bytes);
  for (uint32_t i = tid; i < a.a_bytes / 4; i += NT) A[i] = 0.f;
  if (a.b_resident)
    for (int p = 0; p < 6; ++p) tc_load_factor<NT>(a, p, B + a.pass[p].boff / 4, tid);
  const uint32_t mb = smem_addr(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t baseA = smem_addr(A), baseB = smem_addr(B);
  const int mx = a.md[0], my = a.md[1], mz = a.md[2];
  const int n = a.n, n3 = n * n * n;
  const int64_t groups = (a.Ne + a.G - 1) / a.G;
  uint32_t phase = 0;
  for (int64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int64_t s0 = grp * a.G;
    // gather r_s = R_s r of the group into the layout of pass 0: lines (b, c)
    // numbered b + mp_y c, K = a; one thread per line, four K per store
    {
      const int ka = a.pass[0].ka, L0 = a.pass[0].lines, lbo_w = a.lbo_a / 4;
      const int nox = a.nod[0];
      for (int L = tid; L < a.G * my * mz; L += NT) {
        const int g = L / (my * mz), rem = L - g * (my * mz);
        const int64_t s = s0 + g;
        if (s >= a.Ne) continue;
        const int b = rem % my, c = rem / my;
        const int s32 = (int)s, sxy = s32 / a.nx;
        const int sx = s32 - sxy * a.nx, sy = sxy % a.ny, sz = sxy / a.ny;
        int dy, iy, dz, iz;
        tc_sub_node(b, n, a.nod[1], &dy, &iy);
        tc_sub_node(c, n, a.nod[2], &dz, &iz);
        const int64_t row = (int64_t)a.nx * (tc_wrap(sy + dy, a.ny) + (int64_t)a.ny * tc_wrap(sz + dz, a.nz));
        const int loc = n * (iy + n * iz);
        // node k of the line: left strip k < nox, element nox <= k < nox + n, right strip
        const float* __restrict__ rl = a.r + (tc_wrap(sx - 1, a.nx) + row) * n3 + loc + (n - nox);
        const float* __restrict__ rc = a.r + (sx + row) * n3 + loc;
        const float* __restrict__ rr = a.r + (tc_wrap(sx + 1, a.nx) + row) * n3 + loc;
        const int line = g * L0 + b + a.mp[1] * c;
#pragma unroll 3
        for (int k0 = 0; k0 < mx; k0 += 4) {
          float w[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = k0 + i;
            w[i] = k < nox ? __ldg(rl + k)
                           : (k < nox + n ? __ldg(rc + (k - nox)) : (k < mx ? __ldg(rr + (k - nox - n)) : 0.f));
          }
          *reinterpret_cast<float4*>(A + tc_at<Q>(line, k0, ka, lbo_w)) = tc_tf32x4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    for (int p = 0; p < 6; ++p) {
      const TcPass& ps = a.pass[p];
      if (!a.b_resident) tc_load_factor<NT>(a, p, B, tid);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (tid == 0 && !a.self_test) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t idesc = tc_idesc(ps.np);
        const uint32_t lbo = (uint32_t)a.lbo_a, sbo = (uint32_t)(Q * ps.ka / 4) * lbo, sbo_b = 32u * ps.kp;
        const uint32_t bp = baseB + (a.b_resident ? ps.boff : 0u);
        for (int t = 0; t < ps.tiles; ++t) {
          const uint32_t t0 = (uint32_t)(t == ps.tiles - 1 ? ps.last0 : t * kTcRows);
          for (int i = 0; i < Q; ++i)
            for (int j = 0; j < ps.kp / 8; ++j)
              tc_mma(tmem + (uint32_t)((Q * t + i) * ps.np),
                     tc_desc(baseA + (t0 / 8u) * sbo + (uint32_t)(i * ps.ka / 4 + 2 * j) * lbo, lbo, sbo),
                     tc_desc(bp + 256u * j, 128, sbo_b), idesc, j > 0 ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                     : "memory");
      }
      // one thread waits for the MMAs (the others sleep in the barrier, issuing nothing)
      if (tid == 0 && !tc_wait(mb, phase, a.wait_cycles)) {
        atomicExch(a.status + 1, kDevTimeout);
        abort_flag = 1;
        pending_phase = phase;
      }
      phase ^= 1u;
      __syncthreads();
      const bool ok = abort_flag == 0;
      asm volatile("tcgen05.fence::after_thread_sync;");
      switch (p) {
        case 0: tc_writeback<0, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
        case 1: tc_writeback<1, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
        case 2: tc_writeback<2, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
        case 3: tc_writeback<3, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
        case 4: tc_writeback<4, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
        default: tc_writeback<5, Q, NT>(a, A, tmem, warp, lane, s0, ok); break;
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (abort_flag) break;
    }
    if (abort_flag) break;
  }
  // After a timeout with MMAs issued, they may still be writing the tensor
  // memory about to be freed: one more bounded wait for their commit.  (If it
  // also runs out, the tensor memory's contents are undefined; the status word
  // already tells the host, and the solve reports MG_ECUDA.)
  if (tid == 0 && abort_flag && !a.self_test) tc_wait(mb, pending_phase, a.wait_cycles);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
}

int round_up(int v, int q) { return (v + q - 1) / q * q; }

// Pass shapes and buffer sizes for G subdomains per group and Q lines per
// row; returns the bytes of shared memory the kernel needs (factors resident
// when they fit in `limit`, else one factor at a time).
uint32_t make_plan(TcArgs& a, int G, int Q, int lbo, uint32_t limit) {
  a.G = G;
  a.q = Q;
  a.lbo_a = lbo;
  for (int d = 0; d < 3; ++d) a.mp[d] = round_up(a.md[d], 4);
  // lines of each pass, fast index first: (b, c), (c, px), (q, px), (q, px), (px, c), (b, c)
  const int fast[6] = {a.mp[1], a.mp[2], a.mp[1], a.mp[1], a.mp[0], a.mp[1]};
  const int slow[6] = {a.md[2], a.md[0], a.md[0], a.md[0], a.md[2], a.md[2]};
  uint32_t abytes = 0, bmax = 0, btot = 0;
  int cols = 0;
  for (int p = 0; p < 6; ++p) {
    TcPass& ps = a.pass[p];
    ps.dir = kPassDir[p];
    const int m = a.md[ps.dir];
    ps.fast = fast[p];
    ps.lines = fast[p] * slow[p];
    ps.ka = round_up(m, 4);
    ps.kp = round_up(m, 8);
    ps.np = round_up(m, 16);
    ps.quads = G * ps.lines / Q;
    ps.tiles = (ps.quads + kTcRows - 1) / kTcRows;
    const int rows = std::max(round_up(ps.quads, 8), kTcRows);  // rows the buffer holds
    ps.last0 = rows - kTcRows;
    ps.boff = btot;
    abytes = std::max<uint32_t>(abytes, (uint32_t)(rows / 8) * (uint32_t)(Q * ps.ka / 4) * (uint32_t)lbo);
    const uint32_t fb = (uint32_t)ps.np * ps.kp * 4u;
    bmax = std::max(bmax, fb);
    btot += fb;
    cols = std::max(cols, ps.tiles * Q * ps.np);
  }
  abytes += (uint32_t)lbo;  // the spare core matrix the last row group's K_pad > K_a reads (zero)
  a.a_bytes = abytes;
  a.tmem_cols = 32;
  while ((int)a.tmem_cols < cols) a.tmem_cols *= 2;
  a.b_resident = abytes + btot <= limit ? 1 : 0;
  return abytes + (a.b_resident ? btot : bmax);
}

}  // namespace

namespace {

// Fills the level's arguments and picks the launch shape; false if the
// level's tiles do not fit the kernel's shared and tensor memory.
bool tc_configure(const mg_ctx* c, int l, const float* r, TcArgs& a, int& per_sm, uint32_t& smem) {
  const LevelInfo& lv = c->lev[l];
  a.tab = c->ws.tab32;
  a.r = r;
  a.corr = static_cast<float*>(c->ws.corr);
  a.status = c->ws.status;
  a.Ne = c->Ne;
  a.nx = c->ne[0];
  a.ny = c->ne[1];
  a.nz = c->ne[2];
  a.n = lv.n;
  for (int d = 0; d < 3; ++d) {
    a.md[d] = lv.m[d];
    a.nod[d] = lv.no[d];
    a.S[d] = lv.t[d].S;
    a.SW[d] = lv.t[d].SW;
  }
  a.dinvp = lv.dinvp;
  // Four lines per row of A if the pass outputs fit the tensor memory that
  // way, else two; then the most CTAs per SM (4, 2, 1) whose share of tensor
  // and shared memory holds at least one subdomain (with the bank-spread
  // layout if it fits); within that the group size with the fullest tiles, no
  // larger than needed to give every CTA slot two groups.
  const uint32_t kSmemPerSm = 227 * 1024;
  int G = 0, Q = 4, lbo = 0;
  per_sm = 0;
  smem = 0;
  for (int q : {4, 2}) {
    for (int ctas : {4, 2, 1}) {
      const uint32_t limit = kSmemPerSm / ctas - 1024;
      const uint32_t tlimit = 512u / ctas;
      const int64_t slots = 152LL * ctas;
      const int gmax = (int)std::min<int64_t>(32, std::max<int64_t>(1, (c->Ne + 2 * slots - 1) / (2 * slots)));
      for (int lb : {144, 128}) {
        double best = 0.0;
        for (int g = 1; g <= gmax; ++g) {
          const uint32_t need = make_plan(a, g, q, lb, limit);
          if (a.tmem_cols > tlimit || need > limit) continue;
          int tiles = 0;
          for (int p = 0; p < 6; ++p) tiles = std::max(tiles, a.pass[p].tiles);
          const double fill = (double)g / tiles;  // subdomains per tile of the largest pass
          if (fill >= best) {
            best = fill;
            G = g;
            Q = q;
            per_sm = ctas;
            smem = need;
            lbo = lb;
          }
        }
        if (G > 0) break;
      }
      if (G > 0) break;
    }
    if (G > 0) break;
  }
  if (G == 0) return false;
  make_plan(a, G, Q, lbo, kSmemPerSm / per_sm - 1024);
  return true;
}

}  // namespace

bool fdm_tc_fits(const mg_ctx* c, int l) {
  TcArgs a;
  int per_sm = 0;
  uint32_t smem = 0;
  return l >= 1 && l <= c->L && tc_configure(c, l, nullptr, a, per_sm, smem);
}

cudaError_t launch_fdm_tc(const mg_ctx* c, int l, const float* r, int self_test) {
  TcArgs a;
  int per_sm = 0;
  uint32_t smem = 0;
  if (!tc_configure(c, l, r, a, per_sm, smem)) return cudaErrorNotSupported;
  a.self_test = self_test;
  a.wait_cycles = self_test ? kTcSelfTestWaitCycles : kTcWaitCycles;
  const int G = a.G;
  const bool wide = per_sm == 1;
  auto* kern = a.q == 4 ? (wide ? k_fdm_tc<4, kTcThreadsWide> : k_fdm_tc<4, kTcThreads>)
                        : (wide ? k_fdm_tc<2, kTcThreadsWide> : k_fdm_tc<2, kTcThreads>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (c->Ne + G - 1) / G;
  const int blocks = (int)std::min<int64_t>(groups, 152LL * per_sm);
  launch_pdl(kern, blocks, wide ? kTcThreadsWide : kTcThreads, smem, c->stream, a);
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace mgdg
