// Pass 1 of the dexel offset (Sec. 3.3, the extrusion along x) as a gather.
//
// S_mid(i, j) is the union of the columns i' = i - R .. i + R of row j, every height z
// labelled with the distance dx = |i - i'| of the nearest of them that contains z (the
// closest parent gives the largest residual radius in pass 2).  Written as a partition:
// between consecutive distinct endpoint heights v_k < v_{k+1} the open interval has the label
// O_k = min { |i - i'| : a segment of i' contains (v_k, v_{k+1}) }, the height v_k itself the
// label P_k <= min(O_{k-1}, O_k); the pieces are the maximal runs of equal O labels (closed)
// and the points [v_k, v_k] where P_k is below both neighbours (a zero-length segment, or
// the touching end of a nearer one), at which a run through v_k is split.
//
// GB300 mapping: a block takes a tile of consecutive output columns of row j; the endpoint
// events of the tile's window (tc + 2R source columns, contiguous in the row-major input) are
// staged in shared memory and sorted once by (height, open before close).  A warp then walks
// the sorted events for one output column: the set of open sources is a bit mask (bit
// i' - i + R; one 64-bit word for R < 32, two up to R = 63, four up to 127) kept by an XOR
// scan over the lanes, the nearest open source is found from the mask with find-first-set,
// and the group values O, P and the run starts follow from segmented scans.  The pieces go
// to a per-warp
// buffer in shared memory and are copied out once the column's count has reserved its place
// (a column with more pieces than the buffer is walked a second time, straight into place).
#pragma once
#include "gather2.cuh"

namespace dexel {


constexpr unsigned kEvNone = 0xFFFFFFFFu;  // sentinel payload (sorts last)
constexpr int kNoLabel = 255;

template <typename T>
DXI ukey event_key(T x) { return dkey((double)x); }

template <typename K>
DXI K key_out(ukey u);
template <>
DXI ukey key_out<ukey>(ukey u) { return u; }
template <>
DXI float key_out<float>(ukey u) { return (float)dval(u); }

// The open sources of a window as a bit mask of NW 64-bit words (bit b = source i - R + b).
template <int NW>
struct Mask {
  ukey w[NW];
};

// min |b - R| over the set bits b of the mask (the nearest open source), R < 64 NW / 2
template <int NW>
DXI int nearest_label(const Mask<NW>& m, int R) {
  int best = kNoLabel;
#if defined(__CUDA_ARCH__)
  const int wr = R >> 6, br = R & 63;
  // upwards: the lowest set bit >= R
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    if (q < wr || best != kNoLabel) continue;
    const ukey v = q == wr ? (m.w[q] & (~0ULL << br)) : m.w[q];
    if (v) best = 64 * q + (__ffsll((long long)v) - 1) - R;
  }
  // downwards: the highest set bit <= R
  bool found = false;
#pragma unroll
  for (int q = NW - 1; q >= 0; --q) {
    if (q > wr || found) continue;
    const ukey v = q == wr ? (m.w[q] & (br >= 63 ? ~0ULL : ((2ULL << br) - 1))) : m.w[q];
    if (v) {
      const int d = R - (64 * q + 63 - __clzll((long long)v));
      best = d < best ? d : best;
      found = true;
    }
  }
#endif
  return best;
}

// Walks the sorted events ek/ep[0, E) for output column i (sources s0 + q, payload
// (close << 16) | q); returns the number of S_mid pieces.  With oa != null the pieces with
// index < cap are written at oa, ob, ol (a, b, dx).
template <typename T, int NW>
DXI int column_partition(const Lanes& L, const ukey* ek, const unsigned* ep, int E, int s0,
                         int i, int R, typename H<T>::K* oa, typename H<T>::K* ob, short* ol,
                         int cap, Counters* dctr = nullptr) {
  typedef typename H<T>::K Key;
  Mask<NW> m;  // open sources before the chunk
#pragma unroll
  for (int q = 0; q < NW; ++q) m.w[q] = 0;
  int carry_p = kNoLabel, carry_ob = kNoLabel;  // segmented values of a group that continues
  int carry_o = kNoLabel;  // the label after the previous chunk's last event
  ukey carry_key = 0;
  int cum = 0;
  for (int base = 0; base < E; base += 32) {
    const int t = base + L.lane;
    const bool valid = t < E;
    const ukey key = valid ? ek[t] : ~0ULL;
    const unsigned pay = valid ? ep[t] : kEvNone;
    const bool ev = valid && pay != kEvNone;
    const int b = (int)(pay & 0xFFFFu) + s0 - i + R;
    const bool close = (pay >> 16) & 1u;
    const bool inwin = ev && b >= 0 && b <= 2 * R;
    Mask<NW> tg, M;  // this event's toggle; the open sources after it
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      tg.w[q] = inwin && (b >> 6) == q ? (1ULL << (b & 63)) : 0ULL;
      ukey x = tg.w[q];
#if defined(__CUDA_ARCH__)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const ukey y = __shfl_up_sync(0xffffffffu, x, o);
        if (L.lane >= o) x ^= y;
      }
#endif
      M.w[q] = m.w[q] ^ x;
    }
    // the label after each event: at a group's last event, the label O of the open interval
    // above the group; after the event before it, the label below the group
    const int oab = valid ? nearest_label<NW>(M, R) : kNoLabel;
    ukey prevk = 0;
    int obelow = kNoLabel;
#if defined(__CUDA_ARCH__)
    prevk = __shfl_up_sync(0xffffffffu, key, 1);
    obelow = __shfl_up_sync(0xffffffffu, oab, 1);
#endif
    if (L.lane == 0) {
      prevk = carry_key;
      obelow = carry_o;
    }
    // groups of equal height
    const bool head = valid && (t == 0 || key != prevk);
    const bool last = valid && (t + 1 >= E || ek[t + 1] != key);
    int vp = kNoLabel;   // the group's point label (a single event: not below its neighbours)
    int vob = obelow;    // the label below the group
#if defined(DEXEL_PHASES) && defined(__CUDA_ARCH__)
    if (dctr && L.lane == 0) atomicAdd(&dctr->phase[8], 1ULL);
#endif
    if (w_any(valid && !(head && last))) {
#if defined(DEXEL_PHASES) && defined(__CUDA_ARCH__)
      if (dctr && L.lane == 0) atomicAdd(&dctr->phase[9], 1ULL);
#endif
      // some group has several events (or continues across chunks): the point label is the
      // minimum over the group of the label at the height itself (after an open, before a
      // close), and the label below is the head's; segmented scans, carried into the chunk
      // when the group continues
      int pl = kNoLabel;
      if (inwin) {
        Mask<NW> pm;
#pragma unroll
        for (int q = 0; q < NW; ++q) pm.w[q] = close ? (M.w[q] | tg.w[q]) : M.w[q];
        pl = nearest_label<NW>(pm, R);
      }
      // the group's first lane in this chunk: the last head at or below this lane (none: the
      // group continues from the previous chunk)
#if defined(__CUDA_ARCH__)
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      const unsigned below = hm & (0xffffffffu >> (31 - L.lane));
      const int hl = below ? 31 - __clz((int)below) : -1;
      const int ob_head = __shfl_sync(0xffffffffu, obelow, hl < 0 ? 0 : hl);
      vob = hl >= 0 ? ob_head : carry_ob;
      const int seg0 = hl >= 0 ? hl : 0;
      vp = pl;
      if (hl < 0) vp = vp < carry_p ? vp : carry_p;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int p2 = __shfl_up_sync(0xffffffffu, vp, o);
        if (L.lane - o >= seg0) vp = p2 < vp ? p2 : vp;
      }
#endif
    }
    int here = 0;
    bool pt = false, endrun = false, strun = false;
    int Ok = kNoLabel;
    if (last) {
      Ok = oab;
      const int Om = vob;
      pt = vp < (Om < Ok ? Om : Ok);
      endrun = Om < kNoLabel && (Ok != Om || pt);
      strun = Ok < kNoLabel && (Ok != Om || pt);
      here = (pt ? 1 : 0) + (strun ? 1 : 0);
    }
    const int inc = w_incl_add(here, L.lane);
    const int slot = cum + inc - here;
    if (oa && last) {
      if (endrun && slot - 1 < cap) ob[slot - 1] = key_out<Key>(key);
      if (pt && slot < cap) {
        oa[slot] = key_out<Key>(key);
        ob[slot] = key_out<Key>(key);
        ol[slot] = (short)vp;
      }
      const int s2 = slot + (pt ? 1 : 0);
      if (strun && s2 < cap) {
        oa[s2] = key_out<Key>(key);
        ol[s2] = (short)Ok;
      }
    }
    cum += w_bcast(inc, 31);
#if defined(__CUDA_ARCH__)
#pragma unroll
    for (int q = 0; q < NW; ++q) m.w[q] = __shfl_sync(0xffffffffu, M.w[q], 31);
    carry_p = __shfl_sync(0xffffffffu, vp, 31);
    carry_o = __shfl_sync(0xffffffffu, oab, 31);
    carry_ob = __shfl_sync(0xffffffffu, vob, 31);
    carry_key = __shfl_sync(0xffffffffu, key, 31);
#endif
  }
  return cum;
}

// mask words for a reach: 2R + 1 bits
DXI int mask_words(int R) { return R < 32 ? 1 : (R < 64 ? 2 : 4); }

// Shared memory: sorted events (key, payload), the window's event offsets and per warp a
// buffer of obuf output pieces.
template <typename T>
DXI long long p1g_layout(int tc, int R, int ecap, int obuf, int nwarps, long long* o_off,
                         long long* o_buf) {
  typedef typename H<T>::K Key;
  long long x = (long long)ecap * (sizeof(ukey) + sizeof(unsigned));
  *o_off = x;
  x += (long long)(tc + 2 * R + 2) * sizeof(int);
  x = (x + 15) & ~15LL;
  *o_buf = x;
  x += (long long)nwarps * obuf * (2 * sizeof(Key) + sizeof(short));
  return x + 16;
}

// One tile of k_pass1g: columns i0 .. i0 + tc - 1 of row j (tile = j * tiles_per_row +
// i0 / tc); smem holds the layout p1g_layout(tc, K, ecap, obuf, warps).
template <typename T, int NW>
__device__ __forceinline__ void pass1g_tile(const P1Params<T>& P, long long tile, int tc,
                                            int ecap, int obuf, unsigned char* smem,
                                            ArenaCursor& cur) {
  typedef typename H<T>::K Key;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwb = blockDim.x >> 5;
  long long o_off, o_buf;
  p1g_layout<T>(tc, P.K, ecap, obuf, nwb, &o_off, &o_buf);
  ukey* ek = (ukey*)smem;
  unsigned* ep = (unsigned*)(ek + ecap);
  int* eoff = (int*)(smem + o_off);
  Key* wbuf_a = (Key*)(smem + o_buf);
  Key* wbuf_b = wbuf_a + (long long)nwb * obuf;
  short* wbuf_l = (short*)(wbuf_b + (long long)nwb * obuf);
  const Lanes L{lane, 32};
  const int R = P.K;
  const int tpr = (P.nx + tc - 1) / tc;
  const int j = (int)(tile / tpr);
  const int i0 = (int)(tile % tpr) * tc;
  const int i1 = min(P.nx, i0 + tc);
  const int s0 = max(0, i0 - R), s1 = min(P.nx, i1 + R);
  const int ns = s1 - s0;
  const long long rb = (long long)j * P.nx;
  __syncthreads();
  if (warp == 0) {
    int carry = 0;
    for (int base = 0; base < ns; base += 32) {
      const int q = base + lane;
      int v = 0;
      if (q < ns) {
        const int n = P.col_off[rb + s0 + q + 1] - P.col_off[rb + s0 + q];
        v = P.erode ? 2 * (n + 1) : 2 * n;
      }
      const int inc = w_incl_add(v, lane);
      if (q < ns) eoff[q] = carry + inc - v;
      carry += w_bcast(inc, 31);
    }
    if (lane == 0) eoff[ns] = carry;
  }
  __syncthreads();
  for (int ia = i0; ia < i1;) {
    const int qa = max(0, ia - R) - s0;
    int ib = i1;
    while (ib > ia + 1 && eoff[min(P.nx, ib + R) - s0] - eoff[qa] > ecap) --ib;
    const int qe = min(P.nx, ib + R) - s0;
    const int e0 = eoff[qa];
    const int E = eoff[qe] - e0;
    if (E > ecap) {  // one column's window holds more events than fit: the sweep takes over
      if (threadIdx.x == 0) {
        set_status(&P.ctr->status, ST_OVERFLOW_SLOT);
        P.m_start[(long long)ia * P.ny + j] = -1;  // marks the column (count 0)
        P.m_cnt[(long long)ia * P.ny + j] = 0;
      }
      ia = ib;
      continue;
    }
    int n2 = 1;
    while (n2 < E) n2 <<= 1;
    // stage the events of sources qa .. qe - 1, one thread per source
    for (int q = qa + threadIdx.x; q < qe; q += blockDim.x) {
      const long long c = rb + s0 + q;
      const int g0 = P.col_off[c], g1 = P.col_off[c + 1];
      int o = eoff[q] - e0;
      const int oend = eoff[q + 1] - e0;
      const unsigned src = (unsigned)q;
      if (!P.erode) {
        for (int g = g0; g < g1; ++g) {
          ek[o] = event_key(P.z[2LL * g]);
          ep[o++] = src;
          ek[o] = event_key(P.z[2LL * g + 1]);
          ep[o++] = (1u << 16) | src;
        }
      } else {
        // closure of the complement: (-inf, a0], [b0, a1], ..., [b_last, +inf); zero-length
        // segments leave no gap
        ukey lo = KEY_NINF;
        for (int g = g0; g < g1; ++g) {
          const ukey a = event_key(P.z[2LL * g]), b = event_key(P.z[2LL * g + 1]);
          if (a == b) continue;
          ek[o] = lo;
          ep[o++] = src;
          ek[o] = a;
          ep[o++] = (1u << 16) | src;
          lo = b;
        }
        ek[o] = lo;
        ep[o++] = src;
        ek[o] = KEY_PINF;
        ep[o++] = (1u << 16) | src;
      }
      for (; o < oend; ++o) { ek[o] = ~0ULL; ep[o] = kEvNone; }
    }
    for (int t = E + threadIdx.x; t < n2; t += blockDim.x) { ek[t] = ~0ULL; ep[t] = kEvNone; }
    __syncthreads();
    PHASE_BEGIN();
    // block bitonic sort by (height, open before close)
    for (int k = 2; k <= n2; k <<= 1) {
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int t = threadIdx.x; t < n2; t += blockDim.x) {
          const int x = t ^ jj;
          if (x > t) {
            const bool up = (t & k) == 0;
            const ukey kt = ek[t], kx = ek[x];
            const unsigned pt = ep[t], px = ep[x];
            const bool gt = kt > kx || (kt == kx && (pt >> 16) > (px >> 16));
            if (gt == up) {
              ek[t] = kx; ek[x] = kt;
              ep[t] = px; ep[x] = pt;
            }
          }
        }
        __syncthreads();
      }
    }
    PHASE(0);
    // output columns of the run: pieces go to the warp's buffer, then to the arena; a column
    // with more pieces than the buffer holds is walked a second time straight into the arena
    for (int i = ia + warp; i < ib; i += nwb) {
      Key* ba = wbuf_a + (long long)warp * obuf;
      Key* bb = wbuf_b + (long long)warp * obuf;
      short* bl = wbuf_l + (long long)warp * obuf;
      const int n = column_partition<T, NW>(L, ek, ep, E, s0, i, R, ba, bb, bl, obuf, P.ctr);
      PHASE(1);
      const long long s = arena_take(L, &P.ctr->arena_top[1], P.blk, cur, n);
      const bool fits = s + n <= P.m_cap;
      if (fits && n > 0) {
        if (n <= obuf) {
          for (int q = lane; q < n; q += 32) { P.m_a[s + q] = ba[q]; P.m_b[s + q] = bb[q]; P.m_l[s + q] = bl[q]; }
        } else {
          column_partition<T, NW>(L, ek, ep, E, s0, i, R, P.m_a + s, P.m_b + s, P.m_l + s, 1 << 30);
        }
      }
      if (lane == 0) {
        if (!fits) set_status(&P.ctr->status, ST_OVERFLOW_ARENA);
        const long long q = (long long)i * P.ny + j;
        P.m_start[q] = fits ? s : 0;
        P.m_cnt[q] = n;
        cur.tally += n;
        cur.tmax = n > cur.tmax ? n : cur.tmax;
        PHASE_COUNT(10, 1);
        PHASE_COUNT(11, E);
        PHASE_COUNT(12, n > obuf ? 1 : 0);
      }
      wsync();
      PHASE(2);
    }
    __syncthreads();
    PHASE(3);
    ia = ib;
  }
}

}  // namespace dexel
