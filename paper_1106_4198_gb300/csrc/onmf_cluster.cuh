// Cluster h-solve of the mixed-precision path (the h step of Algorithm 1,
// arXiv:1106.4198, with the multiplicative update of Section 2.1 and the
// exponent gamma; BF16 products, FP32 ratios and h).
//
// A thread-block cluster of C CTAs (C in {1, 2, 4, 8}) solves a tile of 32
// frames. CTA r of the cluster holds the rows [16 mt0(r), 16 mt1(r)) of W in
// shared memory (bf16, row f = row f of W), so W is read from HBM/L2 once
// per minibatch per CTA and each W fragment in shared memory feeds four
// m16n8k16 products (32 frames) instead of one. Per inner iteration:
//   step A  every CTA computes x = eps + W h for its rows and all 32 frames,
//           then p = y/x^2, q = 1/x (FP32) for those rows, rounded to bf16
//           and stored transposed as the operand [P | Q]^T;
//   step B  every CTA forms its partial [W^T p | W^T q] over its rows (the
//           contraction over f is split across the cluster) and stores each
//           partial into the shared memory of the CTA that owns the frame
//           (CTA r owns frames [32r/C, 32(r+1)/C));
//   update  after a cluster barrier each owner adds the C partials in rank
//           order (deterministic), updates its FP32 h and writes the bf16 h
//           into every CTA's operand buffer; a second cluster barrier ends
//           the iteration.
// Frame sums of the fresh-restart start point (h0_k = sum_f y_f / sum W) are
// combined the same way. Every CTA of a cluster runs the same sequence of
// cluster barriers (the tile list, n_in and the flags are uniform over the
// cluster), so the hardware barrier cannot wait on a CTA that left.
#pragma once

#include "onmf_device.cuh"
#include "onmf_hsolve.cuh"
#include "onmf_kernels.cuh"

namespace onmf {

constexpr int kClTile = 32;         // frames per cluster tile
constexpr int kClMaxC = 8;          // CTAs per cluster at most (portable size)
constexpr int kClMaxMtPerWarp = 3;  // m16 row tiles per warp in step A

struct ClLayout {
    int C, FT, MT, RL, KLD, PLD, YLD, OF;
    unsigned ws, hs, pq, ys, recv, hm, fs, total;  // byte offsets, size
};

__host__ __device__ inline unsigned cl_take(unsigned &o, size_t bytes) {
    const unsigned r = o;
    o = (unsigned)((o + bytes + 127) / 128 * 128);
    return r;
}

// Shared-memory layout of the cluster h-solve for C CTAs per cluster:
//   Ws   RL x KLD bf16     this CTA's rows of W (row f, K contiguous)
//   Hs   32 x KLD bf16     h of the tile's frames (frame rows), operand of x
//   PQs  64 x PLD bf16     rows 0..31 p, rows 32..63 q (frame rows, f cont.)
//   yS   32 x YLD f32      y = eps + v of this CTA's rows
//   recv C x 2 x Kp x OF   partial [W^T p | W^T q] of the owned frames, one
//                          slot per source CTA
//   hm   Kp x OF f32       FP32 h of the owned frames
//   fs   2 x C x 32 f32 frame-sum partials (alternating by tile, so a peer
//        that starts its next tile cannot overwrite sums still being read),
//        then 16 spare words, 8 per-warp losses and 32 frame sums
// The +8 / +4 paddings put the 8 rows of every ldmatrix / stmatrix and the
// ratio reads of a warp in distinct banks.
__host__ __device__ inline ClLayout cl_layout(const Shape &s, int C) {
    ClLayout L;
    L.C = C;
    L.FT = s.Fp16 / 16;
    L.MT = (L.FT + C - 1) / C;
    L.RL = 16 * L.MT;
    L.KLD = s.Kp + 8;
    L.PLD = L.RL + 8;
    L.YLD = L.RL + 4;
    L.OF = kClTile / C;
    unsigned o = 0;
    L.ws = cl_take(o, (size_t)L.RL * L.KLD * 2);
    L.hs = cl_take(o, (size_t)kClTile * L.KLD * 2);
    L.pq = cl_take(o, (size_t)2 * kClTile * L.PLD * 2);
    L.ys = cl_take(o, (size_t)kClTile * L.YLD * 4);
    L.recv = cl_take(o, (size_t)2 * kClTile * s.Kp * 4);
    L.hm = cl_take(o, (size_t)L.OF * s.Kp * 4);
    L.fs = cl_take(o, (size_t)2 * C * kClTile * 4 + 256);
    L.total = o;
    return L;
}

// Whether the cluster h-solve covers the shape with C CTAs per cluster.
__host__ __device__ inline bool cl_supported(const Shape &s, int C) {
    const int FT = s.Fp16 / 16;
    return (C == 1 || C == 2 || C == 4 || C == 8) && C <= FT && s.Kp <= 256 &&
           (FT + C - 1) / C <= kWarps * kClMaxMtPerWarp;
}

// m16 row tiles of W held by CTA `rank`: [mt0, mt0 + nmt).
__host__ __device__ inline void cl_rows(const ClLayout &L, int rank, int &mt0, int &nmt) {
    mt0 = rank * L.FT / L.C;
    nmt = (rank + 1) * L.FT / L.C - mt0;
}

// This CTA's rows of W (bf16, row-major, ld Kp in global) -> Ws.
static __device__ void cl_stage_w(const Shape &s, const ClLayout &L, int rank,
                                  const __nv_bfloat16 *Wrow, unsigned char *smem) {
    int mt0, nmt;
    cl_rows(L, rank, mt0, nmt);
    const int f0 = 16 * mt0, rows = 16 * nmt;
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(smem + L.ws);
    const int cpr = s.Kp / 8;  // 16-byte chunks per row
    for (int i = threadIdx.x; i < rows * cpr; i += kThreads) {
        const int r = i / cpr, c = i - r * cpr;
        const int f = f0 + r;
        const bool ok = f < s.F;
        cp_async16(Ws + r * L.KLD + 8 * c, ok ? Wrow + (long long)f * s.Kp + 8 * c : Wrow,
                   ok ? 16 : 0);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
}

// One 32-frame tile (t.nvalid <= 32 frames) on the cluster; W rows staged.
// seq counts the tiles this cluster has solved (the same on every CTA).
template <int KS>
static __device__ void hsolve_tile_cluster(const Shape &s, const ClLayout &L, int rank, float eps,
                                           float gamma, float sw, const TileJob &t,
                                           unsigned char *smem, int seq, int *err) {
    constexpr int KI = (KS + 3) / 4;  // k16 row tiles of W^T per warp in step B
    const int F = s.F, K = s.K, Kp = s.Kp, C = L.C, OF = L.OF;
    const int KLD = L.KLD, PLD = L.PLD, YLD = L.YLD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3, mi = lane >> 3, r8 = lane & 7;
    int mt0, nmt;
    cl_rows(L, rank, mt0, nmt);
    const int f0 = 16 * mt0, rows = 16 * nmt;
    const int vrows = min(rows, F - f0);  // rows of the slice inside F (>= 1)
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(smem + L.ws);
    __nv_bfloat16 *Hs = reinterpret_cast<__nv_bfloat16 *>(smem + L.hs);
    __nv_bfloat16 *PQs = reinterpret_cast<__nv_bfloat16 *>(smem + L.pq);
    float *yS = reinterpret_cast<float *>(smem + L.ys);
    float *recv = reinterpret_cast<float *>(smem + L.recv);
    float *hM = reinterpret_cast<float *>(smem + L.hm);
    float *fs_base = reinterpret_cast<float *>(smem + L.fs);
    float *fs = fs_base + (seq & 1) * C * kClTile;
    float *lw = fs_base + 2 * C * kClTile + 16;
    float *Sj = lw + kWarps;
    const uint32_t recv_a = smem_u32(recv), hs_a = smem_u32(Hs), fs_a = smem_u32(fs);
    const int jo = rank * OF;  // first frame owned by this CTA
    const int lgOF = 31 - __clz(OF);  // OF is a power of two

    // ---- frames -> yS: y = eps + v on rows inside F, 1 elsewhere and on
    //      frames past the end of the tile. Warp w takes frames w, w + 8, ...
    //      (no index division); all loads are in flight at once (4-byte async
    //      copies: a frame's slice is not 16-byte aligned in general), then
    //      one pass adds eps, checks the values and forms the frame sums.
    for (int j = warp; j < t.nvalid; j += kWarps)
        for (int fl = lane; fl < vrows; fl += 32)
            cp_async4(yS + j * YLD + fl, t.Vt + (long long)j * t.ldv + f0 + fl);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    {
        bool bad = false;
        for (int j = warp; j < kClTile; j += kWarps) {
            float a = 0.f;
            for (int fl = lane; fl < rows; fl += 32) {
                float y = 1.f;
                if (j < t.nvalid && fl < vrows) {
                    const float v = yS[j * YLD + fl];
                    bad |= bad_value(v);
                    y = eps + v;
                }
                yS[j * YLD + fl] = y;
                if (fl < vrows) a += y;
            }
            // fresh restart: frame sums over all of F (each CTA adds its rows)
            if (!t.H_in) {
                a = warp_sum(a);
                if (lane < C)
                    st_cluster_f32(map_rank(fs_a + (uint32_t)(rank * kClTile + j) * 4, lane), a);
            }
        }
        if (bad) flag_error(err, ERR_INPUT);
    }
    // frame sums delivered, and every peer is past its previous tile
    cluster_sync();
    if (!t.H_in && tid < kClTile) {
        float S = 0.f;
        for (int r = 0; r < C; ++r) S += fs[r * kClTile + tid];
        Sj[tid] = S / sw;
    }
    __syncthreads();
    // ---- start point: bf16 operand of all 32 frames in every CTA, FP32 h of
    //      the owned frames in hM (k-major: hM[k * OF + jl])
    for (int j = warp; j < kClTile; j += kWarps) {
        const bool own = j >= jo && j < jo + OF;
        for (int k = lane; k < Kp; k += 32) {
            float h = 0.f;
            if (k < K) {
                if (t.H_in)
                    h = (j < t.nvalid) ? t.H_in[(t.j0 + j) * t.ldh_in + k] : 0.f;
                else
                    h = Sj[j];
            }
            Hs[j * KLD + k] = __float2bfloat16_rn(h);
            if (own) hM[k * OF + (j - jo)] = h;
        }
    }
    __syncthreads();

    float lacc = 0.f;
    const int kg = warp >> 1, ng = warp & 1;  // step B: k16 tiles kg + 4i, p (ng 0) or q
    for (int it = 0;; ++it) {
        const bool last = (it == t.n_in);
        if (last && !t.final_pass) break;
        const bool want_loss =
            t.loss_slot && ((last && t.final_pass && !t.loss_first) || (it == 0 && t.loss_first));
        // ---- step A: x = eps + W h over this CTA's rows, ratios, [P | Q]^T
        for (int ml = warp; ml < nmt; ml += kWarps) {
            float d[4][4];
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) d[n][e] = eps;
            const __nv_bfloat16 *wa = Ws + (16 * ml + r8 + 8 * (mi & 1)) * KLD + 8 * (mi >> 1);
            const __nv_bfloat16 *hb = Hs + (r8 + 8 * (mi >> 1)) * KLD + 8 * (mi & 1);
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                uint32_t a[4], b0[4], b1[4];
                ldmatrix_x4(a, wa + 16 * ks);
                ldmatrix_x4(b0, hb + 16 * ks);
                ldmatrix_x4(b1, hb + 16 * KLD + 16 * ks);
                mma_bf16_16816(d[0], a, b0[0], b0[1]);
                mma_bf16_16816(d[1], a, b0[2], b0[3]);
                mma_bf16_16816(d[2], a, b1[0], b1[1]);
                mma_bf16_16816(d[3], a, b1[2], b1[3]);
            }
            // ratios for this m16 tile; the loss (final pass, or the first X
            // of a batch H step) is a separate instantiation
            auto ratios = [&](auto loss_tag) {
                constexpr bool LOSS = decltype(loss_tag)::value != 0;
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    float pv[4], qv[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int fl = 16 * ml + g + 8 * (e >> 1);
                        const int j = 8 * n + 2 * tq + (e & 1);
                        const float y = yS[j * YLD + fl];
                        const float q = rcp_approx(d[n][e]);
                        const float p = y * q * q;
                        const bool ok = fl < vrows;
                        pv[e] = ok ? p : 0.f;
                        qv[e] = ok ? q : 0.f;
                        if (LOSS && ok && j < t.nvalid) {
                            const float r = y * q;
                            lacc += (r - 1.f) - logf(r);
                        }
                    }
                    stmatrix_x4_trans(PQs + ((mi >> 1) * kClTile + 8 * n + r8) * PLD + 16 * ml +
                                          8 * (mi & 1),
                                      pack_bf16(pv[0], pv[1]), pack_bf16(pv[2], pv[3]),
                                      pack_bf16(qv[0], qv[1]), pack_bf16(qv[2], qv[3]));
                }
            };
            if (want_loss)
                ratios(IntTag<1>{});
            else
                ratios(IntTag<0>{});
        }
        __syncthreads();
        if (last) break;

        // ---- step B: partial [W^T p | W^T q] over this CTA's rows
        {
            float c[KI][4][4];
#pragma unroll
            for (int i = 0; i < KI; ++i)
#pragma unroll
                for (int n = 0; n < 4; ++n)
#pragma unroll
                    for (int e = 0; e < 4; ++e) c[i][n][e] = 0.f;
            const __nv_bfloat16 *wt = Ws + (r8 + 8 * (mi >> 1)) * KLD + 8 * (mi & 1);
            const __nv_bfloat16 *pb = PQs + (ng * kClTile + r8 + 8 * (mi >> 1)) * PLD + 8 * (mi & 1);
            for (int fb = 0; fb < nmt; ++fb) {
                uint32_t a[KI][4], b0[4], b1[4];
#pragma unroll
                for (int i = 0; i < KI; ++i)
                    if (kg + 4 * i < KS) ldmatrix_x4_trans(a[i], wt + 16 * fb * KLD + 16 * (kg + 4 * i));
                ldmatrix_x4(b0, pb + 16 * fb);
                ldmatrix_x4(b1, pb + 16 * PLD + 16 * fb);
#pragma unroll
                for (int i = 0; i < KI; ++i)
                    if (kg + 4 * i < KS) {
                        mma_bf16_16816(c[i][0], a[i], b0[0], b0[1]);
                        mma_bf16_16816(c[i][1], a[i], b0[2], b0[3]);
                        mma_bf16_16816(c[i][2], a[i], b1[0], b1[1]);
                        mma_bf16_16816(c[i][3], a[i], b1[2], b1[3]);
                    }
            }
            // to the owners: recv[src][p|q][k][jl] in the owner's shared
            // memory. Lanes tq and tq^1 swap halves so that each lane holds 4
            // consecutive frames of one k: lane tq even keeps row g (frames
            // 2tq..2tq+3), lane tq odd row g + 8 (frames 2tq-2..2tq+1), and
            // each warp store moves 16 bytes per lane.
            const bool odd = tq & 1;
            const int jq = 2 * (tq & ~1);  // first of the lane's 4 frames within the n8 tile
#pragma unroll
            for (int i = 0; i < KI; ++i)
                if (kg + 4 * i < KS) {
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        // even lanes send (e2, e3), odd lanes send (e0, e1)
                        const float s0 = odd ? c[i][n][0] : c[i][n][2];
                        const float s1 = odd ? c[i][n][1] : c[i][n][3];
                        const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1);
                        const float r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                        float v[4];
                        if (odd) {  // row g + 8: partner's e2, e3 then own e2, e3
                            v[0] = r0; v[1] = r1; v[2] = c[i][n][2]; v[3] = c[i][n][3];
                        } else {    // row g: own e0, e1 then partner's e0, e1
                            v[0] = c[i][n][0]; v[1] = c[i][n][1]; v[2] = r0; v[3] = r1;
                        }
                        const int j = 8 * n + jq;  // frames j..j+3, one owner (OF >= 4)
                        const int o = j >> lgOF, jl = j & (OF - 1);
                        const int k = 16 * (kg + 4 * i) + g + (odd ? 8 : 0);
                        const uint32_t off = (uint32_t)((((rank * 2 + ng) * Kp + k) * OF + jl) * 4);
                        st_cluster_f32x4(map_rank(recv_a + off, o), v[0], v[1], v[2], v[3]);
                    }
                }
        }
        cluster_sync();
        // ---- owners: sum the partials in rank order, update h, broadcast bf16 h
        {
            // the h penalty lambda psi(s~), psi = log(a + s) (Section 2.2,
            // "Extensions"): its tangent at the current h adds
            // lambda / (a + s~) to the denominator, s~ = sum_k h_k of the
            // frame before the step (warp w: owned frames w, w + 8, ...;
            // lanes over k, then a warp sum)
            __shared__ float s_hpen[kClTile];
            const bool hp = t.hpen > 0.f;
            if (hp) {
                for (int jl = warp; jl < OF; jl += kWarps) {
                    float v = 0.f;
                    for (int k = lane; k < Kp; k += 32) v += hM[k * OF + jl];
                    v = warp_sum(v);
                    if (lane == 0) s_hpen[jl] = __fdiv_rn(t.hpen, t.hpen_a + v);
                }
                __syncthreads();
            }
            // thread: one k, 4 consecutive owned frames (OF >= 4)
            const int lg4 = lgOF - 2;
            for (int item = tid; item < (Kp << lg4); item += kThreads) {
                const int k = item >> lg4, jl = (item & ((1 << lg4) - 1)) * 4;
                float4 nm = make_float4(0.f, 0.f, 0.f, 0.f), dn = nm;
                for (int r = 0; r < C; ++r) {
                    const float4 a = *reinterpret_cast<const float4 *>(recv + ((r * 2) * Kp + k) * OF + jl);
                    const float4 b =
                        *reinterpret_cast<const float4 *>(recv + ((r * 2 + 1) * Kp + k) * OF + jl);
                    nm.x += a.x; nm.y += a.y; nm.z += a.z; nm.w += a.w;
                    dn.x += b.x; dn.y += b.y; dn.z += b.z; dn.w += b.w;
                }
                if (hp) {
                    dn.x += s_hpen[jl];
                    dn.y += s_hpen[jl + 1];
                    dn.z += s_hpen[jl + 2];
                    dn.w += s_hpen[jl + 3];
                }
                float4 h = *reinterpret_cast<const float4 *>(hM + k * OF + jl);
                with_gamma_mode(gamma, [&](auto gm) {
                    constexpr int GM = decltype(gm)::value;
                    if (dn.x > 0.f) h.x = scale_pow<GM>(h.x, __fdividef(nm.x, dn.x), gamma);
                    if (dn.y > 0.f) h.y = scale_pow<GM>(h.y, __fdividef(nm.y, dn.y), gamma);
                    if (dn.z > 0.f) h.z = scale_pow<GM>(h.z, __fdividef(nm.z, dn.z), gamma);
                    if (dn.w > 0.f) h.w = scale_pow<GM>(h.w, __fdividef(nm.w, dn.w), gamma);
                });
                *reinterpret_cast<float4 *>(hM + k * OF + jl) = h;
                __nv_bfloat16 *hr = Hs + (jo + jl) * KLD + k;
                hr[0] = __float2bfloat16_rn(h.x);
                hr[KLD] = __float2bfloat16_rn(h.y);
                hr[2 * KLD] = __float2bfloat16_rn(h.z);
                hr[3 * KLD] = __float2bfloat16_rn(h.w);
            }
            __syncthreads();
            // the owned rows of Hs to every peer, 16 bytes per store; warp per row
            const int cpr = Kp / 8;  // <= 32
            for (int row = warp; row < (C - 1) * OF; row += kWarps) {
                const int pi = row >> lgOF, jl = row & (OF - 1);
                const int r = pi + (pi >= rank ? 1 : 0);
                if (lane < cpr) {
                    const uint32_t off = (uint32_t)(((jo + jl) * KLD + 8 * lane) * 2);
                    const uint4 v = *reinterpret_cast<const uint4 *>(Hs + (jo + jl) * KLD + 8 * lane);
                    st_cluster_v4(map_rank(hs_a + off, r), v);
                }
            }
        }
        cluster_sync();
    }

    // ---- outputs
    if (t.loss_slot) {
        const float l = warp_sum(lacc);
        if (lane == 0) lw[warp] = l;
        __syncthreads();
        if (tid == 0) {
            double dsum = 0.0;
            for (int w = 0; w < kWarps; ++w) dsum += (double)lw[w];
            *t.loss_slot = dsum;
        }
    }
    if (t.final_pass && t.Pg) {
        __nv_bfloat16 *Pg = reinterpret_cast<__nv_bfloat16 *>(t.Pg);
        __nv_bfloat16 *Qg = reinterpret_cast<__nv_bfloat16 *>(t.Qg);
        __nv_bfloat16 *Hg = reinterpret_cast<__nv_bfloat16 *>(t.Hg);
        const int cpr = rows / 8;  // 16-byte chunks of a frame's slice
        // P and Q rows of the slice: warp per (p|q, frame) row
        for (int row = warp; row < 2 * kClTile; row += kWarps) {
            const int w = row >> 5, j = row & (kClTile - 1);
            if (j >= t.nvalid) continue;
            __nv_bfloat16 *dst = (w ? Qg : Pg) + (t.j0 + j) * s.Fp16 + f0;
            for (int c = lane; c < cpr; c += 32)
                *reinterpret_cast<uint4 *>(dst + 8 * c) =
                    *reinterpret_cast<const uint4 *>(PQs + row * PLD + 8 * c);
        }
        // H of the owned frames (k rows, frames contiguous), 0 past the tile
        for (int i = tid; i < (Kp << lgOF); i += kThreads) {
            const int k = i >> lgOF, j = jo + (i & (OF - 1));
            if (t.j0 + j < t.betap)
                Hg[(long long)k * t.betap + t.j0 + j] =
                    (j < t.nvalid) ? Hs[j * KLD + k] : __float2bfloat16_rn(0.f);
        }
    }
    if (t.H_out) {
        for (int jl = warp; jl < OF; jl += kWarps) {
            if (jo + jl >= t.nvalid) continue;
            for (int k = lane; k < K; k += 32) t.H_out[(t.j0 + jo + jl) * t.ldh + k] = hM[k * OF + jl];
        }
    }
    __syncthreads();
}

// grid_sync followed by a cluster-wide vote, so that every CTA of a cluster
// takes the same branch (a CTA must not leave while a peer still waits at a
// cluster barrier). vote: two alternating rows of kClMaxC flags.
__device__ __forceinline__ bool cl_grid_sync(unsigned *counter, unsigned nblocks, unsigned &epoch,
                                             int *err, int (*vote)[kClMaxC], int &vp, int C,
                                             int rank) {
    const bool ok = grid_sync(counter, nblocks, epoch, err);
    if ((int)threadIdx.x < C)
        st_cluster_u32(map_rank(smem_u32(&vote[vp][rank]), threadIdx.x), ok ? 1u : 0u);
    cluster_sync();
    bool all = true;
    for (int r = 0; r < C; ++r) all = all && vote[vp][r] != 0;
    vp ^= 1;
    return all;
}

}  // namespace onmf
