// Batched one-sided (Hestenes) Jacobi SVD of the LFA symbols, fused with symbol
// assembly (arXiv 2506.05617, Sec. III: symbol A_k = sum_y M_y exp(2 pi i <k,y>)
// and its SVD A_k = U_k S_k V_k^*, Algorithm 1 lines 4-5).
//
// Design (sm_103a, one symbol per "team group"):
//  * The N columns of X (X = A_k or A_k^*, M x N, N = r) are paired; each pair
//    (p, q) is owned by a team of L lanes, each lane holding MR rows of x_p and
//    x_q (and WR rows of the accumulated rotations w_p, w_q) in registers.
//    Rows are interleaved: lane l holds rows l, l + L, l + 2L, ...
//  * One round: every team forms alpha = |x_p|^2, beta = |x_q|^2,
//    gamma = x_p^* x_q (a butterfly over its L lanes) and applies the complex
//    Jacobi rotation that makes x_p, x_q orthogonal when
//    |gamma| > tol * sqrt(alpha beta). The N/2 pairs of a round are disjoint.
//  * Rounds follow the circle-method round robin (all N(N-1)/2 pairs once per
//    sweep). Teams are relabelled between rounds so that each team keeps one
//    of its columns in registers and receives one through shared memory (half
//    the columns move per round); at a sweep boundary every team reloads its
//    round-0 pair. The schedule table is built on the host at plan time.
//  * Sweeps repeat until no pair of a sweep was rotated (or max_sweeps).
//    Singular values are the final column norms (recomputed, not updated);
//    U (or V for wide symbols) columns are the normalised X columns; the other
//    factor is the accumulated rotation matrix W.
//  * Symbol assembly is fused: each lane assembles its own entries of X from the
//    weights (read through L1/L2) and the k_h x k_w phase grid of the frequency,
//    which is built in shared memory from the fp32 twiddle tables.
//  * Work is pulled from a queue (one atomic ticket per item), so one persistent
//    launch serves all layers of the same variant, with uneven F_h.
#pragma once

#include "lfa_internal.cuh"

namespace lfa {

template <int NP_, int L_, int MR_, int WR_, bool VEC_>
struct JCfg {
  static constexpr int NP = NP_, L = L_, MR = MR_, WR = WR_;
  static constexpr bool VEC = VEC_;
  static constexpr int T = NP * L;               // threads per symbol
  static constexpr int UT = T <= 32 ? 32 : T;    // threads per unit (warp or CTA)
  static constexpr int SPU = T <= 32 ? 32 / T : 1;
  static constexpr int BLOCK = T <= 32 ? 128 : T;
  static constexpr int UPB = BLOCK / UT;         // units per CTA
  static constexpr int NC = 2 * NP;              // column slots (N padded to even)
  static constexpr int XR = MR * L;              // X row capacity
  static constexpr int WRC = WR * L;             // W row capacity (also staged when !VEC? no)
  static constexpr int CS = XR + (VEC ? WRC : 0) + 2;   // mailbox column stride (float2)
  static constexpr int MAILBOX = NC * CS;
  static constexpr size_t SYM_BYTES = (size_t)(MAILBOX + kMaxTaps) * 8 + NC * 4 + 64;
  static constexpr size_t UNIT_BYTES = SPU * SYM_BYTES + 64;
  static constexpr size_t SMEM = UPB * UNIT_BYTES;
};

template <int T>
__device__ __forceinline__ unsigned sym_mask(int sym) {
  if constexpr (T >= 32) return 0xffffffffu;
  else return ((1u << T) - 1u) << ((sym * T) & 31);
}

template <int L>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <class C>
__device__ __forceinline__ void unit_sync() {
  if constexpr (C::UT == 32) __syncwarp();
  else __syncthreads();
}

// Sum over the UT threads of a unit (all threads must call it).
template <class C>
__device__ __forceinline__ float unit_sum(float v, float* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if constexpr (C::UT == 32) {
    return v;
  } else {
    const int wid = (threadIdx.x % C::UT) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[wid] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < C::UT / 32; ++i) s += red[i];
    return s;
  }
}

// Entry X[row][col] of the symbol of frequency (phases in `phs`), or 0 outside M x N.
template <bool FUSED>
__device__ __forceinline__ float2 x_entry(const LayerArgs& La, int h, int row, int col,
                                          const float2* phs, int kk) {
  if (row >= La.M || col >= La.N) return make_float2(0.f, 0.f);
  const int o = La.wide ? col : row;
  const int i = La.wide ? row : col;
  float re = 0.f, im = 0.f;
  if constexpr (FUSED) {
    const float* wp = La.w + ((size_t)o * La.c_in + i) * kk;
    for (int t = 0; t < kk; ++t) {
      const float wv = __ldg(wp + t);
      const float2 p = phs[t];
      re = fmaf(wv, p.x, re);
      im = fmaf(wv, p.y, im);
    }
  } else {
    const float2 v = La.symbols[((size_t)h * La.c_out + o) * La.c_in + i];
    re = v.x;
    im = v.y;
  }
  return make_float2(re, La.wide ? -im : im);
}

template <class C, bool FUSED>
__global__ void __launch_bounds__(C::BLOCK)
jacobi_kernel(const __grid_constant__ JacobiLaunch P) {
  constexpr int NP = C::NP, L = C::L, MR = C::MR, WR = C::WR, T = C::T, NC = C::NC;
  constexpr int Cn = NC - 1;  // rounds per sweep
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int unit = threadIdx.x / C::UT;
  const int ut = threadIdx.x % C::UT;
  const int sym = ut / T;
  const int st = ut % T;
  const int team = st / L;
  const int lane = st % L;
  unsigned char* ubase = smem_raw + (size_t)unit * C::UNIT_BYTES;
  float2* mbox = reinterpret_cast<float2*>(ubase + (size_t)sym * C::SYM_BYTES);
  float2* phs = mbox + C::MAILBOX;
  float* ssig = reinterpret_cast<float*>(phs + kMaxTaps);
  int* ubox = reinterpret_cast<int*>(ubase + (size_t)C::SPU * C::SYM_BYTES);  // item, flags
  float* ured = reinterpret_cast<float*>(ubox + 4);                          // reductions

  Counters* ctr = P.counters;
  unsigned int* queue = &ctr->queue[P.queue_slot];

  for (;;) {
    // ---------------------------------------------------------------- fetch a work item
    int item;
    if constexpr (C::UT == 32) {
      int v = 0;
      if (ut == 0) v = (int)atomicAdd(queue, 1u);
      item = __shfl_sync(0xffffffffu, v, 0);
    } else {
      if (ut == 0) ubox[0] = (int)atomicAdd(queue, 1u);
      __syncthreads();
      item = ubox[0];
      __syncthreads();
    }
    if (item >= P.total_items) break;
    int li = 0;
    while (li + 1 < P.nlayers && item >= P.L[li + 1].item_begin) ++li;
    const LayerArgs& La = P.L[li];
    const int h = (item - La.item_begin) * C::SPU + sym;
    const bool active = h < La.F_h;
    const int kk = La.kh * La.kw;
    const int f = active ? La.half[h] : 0;
    const int jj = f / La.m;
    const int ll = f - jj * La.m;

    // ---------------------------------------------------------------- phases exp(2 pi i <k, y_ab>)
    if constexpr (FUSED) {
      for (int t = st; t < kk; t += T) {
        const int a = t / La.kw, b = t - a * La.kw;
        int ia = (jj * (a - La.ph)) % La.n;
        if (ia < 0) ia += La.n;
        int ib = (ll * (b - La.pw)) % La.m;
        if (ib < 0) ib += La.m;
        const float2 p = La.tw_n[ia], q = La.tw_m[ib];
        phs[t] = make_float2(p.x * q.x - p.y * q.y, p.x * q.y + p.y * q.x);
      }
      unit_sync<C>();
    }

    // ---------------------------------------------------------------- assemble the round-0 pair
    ushort2 cur = P.sched[team];
    int ca = cur.x, cb = cur.y;
    float2 xa[MR], xb[MR];
    float2 wa[C::VEC ? WR : 1], wb[C::VEC ? WR : 1];
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int row = lane + L * i;
      xa[i] = active ? x_entry<FUSED>(La, h, row, ca, phs, kk) : make_float2(0.f, 0.f);
      xb[i] = active ? x_entry<FUSED>(La, h, row, cb, phs, kk) : make_float2(0.f, 0.f);
    }
    if constexpr (C::VEC) {
#pragma unroll
      for (int i = 0; i < WR; ++i) {
        const int row = lane + L * i;
        wa[i] = make_float2(row == ca && row < La.N ? 1.f : 0.f, 0.f);
        wb[i] = make_float2(row == cb && row < La.N ? 1.f : 0.f, 0.f);
      }
    }

    // ---------------------------------------------------------------- sweeps
    const float tol2 = La.tol2;
    int sweeps = 0, nrot = 0;
    bool converged = false;
    for (int sw = 0; sw < P.max_sweeps; ++sw) {
      int rotated = 0;
      for (int rr = 0; rr < Cn; ++rr) {
        float al = 0.f, be = 0.f, gr = 0.f, gi = 0.f;
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          al = fmaf(xa[i].x, xa[i].x, fmaf(xa[i].y, xa[i].y, al));
          be = fmaf(xb[i].x, xb[i].x, fmaf(xb[i].y, xb[i].y, be));
          gr = fmaf(xa[i].x, xb[i].x, fmaf(xa[i].y, xb[i].y, gr));   // Re(conj(xa) xb)
          gi = fmaf(xa[i].x, xb[i].y, fmaf(-xa[i].y, xb[i].x, gi));  // Im(conj(xa) xb)
        }
        al = team_sum<L>(al);
        be = team_sum<L>(be);
        gr = team_sum<L>(gr);
        gi = team_sum<L>(gi);
        const float g2 = fmaf(gr, gr, gi * gi);
        if (g2 > tol2 * (al * be)) {
          // rotation J = [[c, s e], [-s conj(e), c]] with e = gamma/|gamma|, t = tan:
          // t solves t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 |gamma|), |t| <= 1.
          // Applied as x + (c - 1) x + ...: for small t, c rounds to 1 in fp32 and a rotation
          // with c = 1, s = t would grow both norms by t^2/2; c - 1 = -t^2 / (r (1 + r)),
          // r = sqrt(1 + t^2), keeps each rotation norm-preserving to O(eps t^2).
          const float g = sqrtf(g2);
          const float zeta = (be - al) / (2.f * g);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + hypotf(1.f, zeta));
          const float rr2 = sqrtf(fmaf(t, t, 1.f));
          const float cm1 = -(t * t) / (rr2 * (1.f + rr2));
          const float s = t / rr2;
          const float er = gr / g, ei = gi / g;
          const float sr = s * er, si = s * ei;
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            const float2 A = xa[i], B = xb[i];
            xa[i].x = fmaf(cm1, A.x, A.x) - fmaf(sr, B.x, si * B.y);
            xa[i].y = fmaf(cm1, A.y, A.y) - fmaf(sr, B.y, -si * B.x);
            xb[i].x = fmaf(cm1, B.x, B.x) + fmaf(sr, A.x, -si * A.y);
            xb[i].y = fmaf(cm1, B.y, B.y) + fmaf(sr, A.y, si * A.x);
          }
          if constexpr (C::VEC) {
#pragma unroll
            for (int i = 0; i < WR; ++i) {
              const float2 A = wa[i], B = wb[i];
              wa[i].x = fmaf(cm1, A.x, A.x) - fmaf(sr, B.x, si * B.y);
              wa[i].y = fmaf(cm1, A.y, A.y) - fmaf(sr, B.y, -si * B.x);
              wb[i].x = fmaf(cm1, B.x, B.x) + fmaf(sr, A.x, -si * A.y);
              wb[i].y = fmaf(cm1, B.y, B.y) + fmaf(sr, A.y, si * A.x);
            }
          }
          rotated = 1;
          ++nrot;
        }
        // -------------------------------------------------------------- exchange
        const int rn = (rr + 1 == Cn) ? 0 : rr + 1;
        const ushort2 nx = P.sched[rn * NP + team];
        if (rn != 0) {
          // keep-one transition: exactly one of the team's columns stays in its slot
          const bool keep_a = (nx.x == ca);
          float2* dst = mbox + (keep_a ? cb : ca) * C::CS;
#pragma unroll
          for (int i = 0; i < MR; ++i) dst[lane + L * i] = keep_a ? xb[i] : xa[i];
          if constexpr (C::VEC) {
#pragma unroll
            for (int i = 0; i < WR; ++i) dst[C::XR + lane + L * i] = keep_a ? wb[i] : wa[i];
          }
          unit_sync<C>();
          const int in = keep_a ? nx.y : nx.x;
          const float2* src = mbox + in * C::CS;
          if (keep_a) {
#pragma unroll
            for (int i = 0; i < MR; ++i) xb[i] = src[lane + L * i];
            if constexpr (C::VEC) {
#pragma unroll
              for (int i = 0; i < WR; ++i) wb[i] = src[C::XR + lane + L * i];
            }
            cb = in;
          } else {
#pragma unroll
            for (int i = 0; i < MR; ++i) xa[i] = src[lane + L * i];
            if constexpr (C::VEC) {
#pragma unroll
              for (int i = 0; i < WR; ++i) wa[i] = src[C::XR + lane + L * i];
            }
            ca = in;
          }
        } else {
          // sweep boundary: every team reloads its round-0 pair
          float2* da = mbox + ca * C::CS;
          float2* db = mbox + cb * C::CS;
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            da[lane + L * i] = xa[i];
            db[lane + L * i] = xb[i];
          }
          if constexpr (C::VEC) {
#pragma unroll
            for (int i = 0; i < WR; ++i) {
              da[C::XR + lane + L * i] = wa[i];
              db[C::XR + lane + L * i] = wb[i];
            }
          }
          unit_sync<C>();
          ca = nx.x;
          cb = nx.y;
          const float2* sa = mbox + ca * C::CS;
          const float2* sb = mbox + cb * C::CS;
#pragma unroll
          for (int i = 0; i < MR; ++i) {
            xa[i] = sa[lane + L * i];
            xb[i] = sb[lane + L * i];
          }
          if constexpr (C::VEC) {
#pragma unroll
            for (int i = 0; i < WR; ++i) {
              wa[i] = sa[C::XR + lane + L * i];
              wb[i] = sb[C::XR + lane + L * i];
            }
          }
        }
      }
      ++sweeps;
      // a symbol has converged when none of its pairs rotated in this sweep
      bool any_sym, any_unit;
      if constexpr (C::UT == 32) {
        const unsigned bal = __ballot_sync(0xffffffffu, rotated != 0);
        any_sym = (bal & sym_mask<T>(sym)) != 0u;
        any_unit = bal != 0u;
      } else {
        any_unit = __syncthreads_or(rotated) != 0;
        any_sym = any_unit;
      }
      if (!any_sym && !converged) {
        converged = true;
        if (st == 0 && active) atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      }
      if (!any_unit) break;
    }
    if (!converged && st == 0 && active) {
      atomicAdd(&ctr->sweeps, (unsigned long long)sweeps);
      atomicAdd(&ctr->unconverged, 1ull);
    }
    if (lane == 0 && nrot && active) atomicAdd(&ctr->rotations, (unsigned long long)nrot);

    // ---------------------------------------------------------------- singular values, order
    float al = 0.f, be = 0.f;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      al = fmaf(xa[i].x, xa[i].x, fmaf(xa[i].y, xa[i].y, al));
      be = fmaf(xb[i].x, xb[i].x, fmaf(xb[i].y, xb[i].y, be));
    }
    al = team_sum<L>(al);
    be = team_sum<L>(be);
    float sa = sqrtf(al), sb = sqrtf(be);
    float nwa = 1.f, nwb = 1.f;  // norms of the accumulated rotation columns (1 up to rounding)
    if constexpr (C::VEC) {
      float qa = 0.f, qb = 0.f;
#pragma unroll
      for (int i = 0; i < WR; ++i) {
        qa = fmaf(wa[i].x, wa[i].x, fmaf(wa[i].y, wa[i].y, qa));
        qb = fmaf(wb[i].x, wb[i].x, fmaf(wb[i].y, wb[i].y, qb));
      }
      qa = team_sum<L>(qa);
      qb = team_sum<L>(qb);
      // x_p = A w_p exactly up to rounding, so sigma_p = |x_p| / |w_p| with v_p = w_p / |w_p|
      nwa = qa > 0.f ? sqrtf(qa) : 1.f;
      nwb = qb > 0.f ? sqrtf(qb) : 1.f;
      sa = sa / nwa;
      sb = sb / nwb;
    }
    const int N = La.N, M = La.M;
    if (lane == 0) {
      if (ca < N) ssig[ca] = sa;
      if (cb < N) ssig[cb] = sb;
    }
    unit_sync<C>();
    int rka = 0, rkb = 0;
    bool finite = true;
    for (int q = 0; q < N; ++q) {
      const float v = ssig[q];
      finite = finite && isfinite(v);
      rka += (v > sa) || (v == sa && q < ca);
      rkb += (v > sb) || (v == sb && q < cb);
    }
    if (active && st == 0 && !finite) atomicAdd(&ctr->nonfinite, 1ull);
    if (active && lane == 0) {
      const int r = La.r;
      float* row = La.sigma + (size_t)(P.half_output ? h : f) * r;
      if (ca < N) row[rka] = sa;
      if (cb < N) row[rkb] = sb;
      if (!P.half_output) {
        const int fc = ((La.n - jj) % La.n) * La.m + (La.m - ll) % La.m;
        if (fc != f) {
          float* rowc = La.sigma + (size_t)fc * r;
          if (ca < N) rowc[rka] = sa;
          if (cb < N) rowc[rkb] = sb;
        }
      }
    }

    if constexpr (C::VEC) {
      // -------------------------------------------------------------- stage U / V by rank
      // normalised X columns -> mailbox column `rank` rows [0, XR); W columns -> rows [XR, XR+WRC)
      int* defc = ubox + 1;  // count of zero columns of this unit's symbols (any symbol)
      if (ut == 0) *defc = 0;
      unit_sync<C>();
      const bool za = !(sa >= 1e-30f), zb = !(sb >= 1e-30f);   // zero (or NaN) column
      const float ia = za ? 0.f : 1.f / sqrtf(al), ib = zb ? 0.f : 1.f / sqrtf(be);
      const float iwa = 1.f / nwa, iwb = 1.f / nwb;
      if (ca < N) {
        float2* d = mbox + rka * C::CS;
#pragma unroll
        for (int i = 0; i < MR; ++i) d[lane + L * i] = make_float2(xa[i].x * ia, xa[i].y * ia);
#pragma unroll
        for (int i = 0; i < WR; ++i) d[C::XR + lane + L * i] = make_float2(wa[i].x * iwa, wa[i].y * iwa);
        if (za && lane == 0) { ssig[ca] = -1.f; atomicAdd(defc, 1); }
      }
      if (cb < N) {
        float2* d = mbox + rkb * C::CS;
#pragma unroll
        for (int i = 0; i < MR; ++i) d[lane + L * i] = make_float2(xb[i].x * ib, xb[i].y * ib);
#pragma unroll
        for (int i = 0; i < WR; ++i) d[C::XR + lane + L * i] = make_float2(wb[i].x * iwb, wb[i].y * iwb);
        if (zb && lane == 0) { ssig[cb] = -1.f; atomicAdd(defc, 1); }
      }
      unit_sync<C>();
      // -------------------------------------------------------------- complete zero columns
      // A zero singular value leaves x_p = 0; its left vector is any unit vector orthogonal to
      // the others: Gram-Schmidt of the canonical vectors e_k against the accepted columns.
      if (*defc > 0) {
        for (int sidx = 0; sidx < C::SPU; ++sidx) {
          float2* mb = reinterpret_cast<float2*>(ubase + (size_t)sidx * C::SYM_BYTES);
          float* sg = reinterpret_cast<float*>(mb + C::MAILBOX + kMaxTaps);
          float2* tmp = mb + C::MAILBOX;  // phases are no longer needed
          const int hh = (item - La.item_begin) * C::SPU + sidx;
          if (hh >= La.F_h) continue;
          // ranks of zero columns: sg[col] == -1; the rank order among them follows col index
          int kstart = 0;
          for (int d = 0; d < N; ++d) {
            // rank d is zero if the column holding rank d has sg == -1; recover by counting
            int zero_cnt = 0;
            for (int q = 0; q < N; ++q) zero_cnt += (sg[q] == -1.f);
            if (d < N - zero_cnt) continue;          // zero columns take the last ranks
            for (int k = kstart; k < M; ++k) {
              float nrm = 0.f;
              for (int row = ut; row < M; row += C::UT) {
                float vr = (row == k) ? 1.f : 0.f, vi = 0.f;
                for (int q = 0; q < N; ++q) {
                  if (q >= N - zero_cnt && q >= d) continue;  // not yet accepted
                  const float2 uq = mb[q * C::CS + row];
                  const float2 uk = mb[q * C::CS + k];
                  // v -= u_q conj(u_q[k])
                  vr -= uq.x * uk.x + uq.y * uk.y;
                  vi -= uq.y * uk.x - uq.x * uk.y;
                }
                tmp[row] = make_float2(vr, vi);
                nrm += vr * vr + vi * vi;
              }
              nrm = unit_sum<C>(nrm, ured);
              if (nrm > 0.25f) {
                const float inv = 1.f / sqrtf(nrm);
                for (int row = ut; row < M; row += C::UT)
                  mb[d * C::CS + row] = make_float2(tmp[row].x * inv, tmp[row].y * inv);
                kstart = k + 1;
                unit_sync<C>();
                break;
              }
              unit_sync<C>();
            }
          }
        }
        unit_sync<C>();
      }
      // -------------------------------------------------------------- coalesced write-out
      if (active) {
        float2* Xo = La.wide ? La.V : La.U;     // normalised X columns
        float2* Wo = La.wide ? La.U : La.V;     // accumulated rotations
        float2* xo = Xo + (size_t)h * M * N;
        for (int e = st; e < M * N; e += T) {
          const int row = e / N, s = e - row * N;
          xo[e] = mbox[s * C::CS + row];
        }
        float2* wo = Wo + (size_t)h * N * N;
        for (int e = st; e < N * N; e += T) {
          const int row = e / N, s = e - row * N;
          wo[e] = mbox[s * C::CS + C::XR + row];
        }
      }
    }
    unit_sync<C>();
  }
}

}  // namespace lfa
