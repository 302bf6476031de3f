// Product plans and the stage order of Alg. 5 (binPolyMul).
#include <algorithm>
#include <cstring>
#include <stdexcept>

#include "kernels.h"
#include "plan.h"

namespace gf2x {

void fill_dev_tables(DevTables *h) {
    const HostTables &H = host_tables();
    static_assert(sizeof(h->S) == sizeof(H.S), "S layout");
    std::memcpy(h->S, H.S, sizeof(H.S));
    for (int p = 0; p < 8; p++)
        for (int v = 0; v < 256; v++) {
            const u128 &x = H.chr_in[p][v];
            h->chr_in[p][v] = make_uint4((uint32_t)x.lo, (uint32_t)(x.lo >> 32), (uint32_t)x.hi,
                                         (uint32_t)(x.hi >> 32));
        }
    std::memcpy(h->mul8, H.mul8, sizeof(H.mul8));
    std::memcpy(h->shfl_basis, H.shfl_basis, sizeof(H.shfl_basis));
    std::memcpy(h->shfl_m4r, H.shfl_m4r, sizeof(H.shfl_m4r));
    // rows 0-2 of contiguous FFT tiles: s_r of index bits 3..7 (per lane) and
    // of bits 8..11 and r+1..2 (per warp), by the linearity of s_r
    auto s_of = [&](int r, uint32_t alpha) {
        uint32_t v = 0;
        for (int t = 0; t < 32; t++)
            if ((alpha >> t) & 1) v ^= H.S[r][t];
        return v;
    };
    for (int x = 0; x < 256; x++)
        for (int l = 0; l < 32; l++) {
            uint32_t w = H.mul8[(0x80 << 8) | x];
            for (int r = 0; r < 3; r++) {
                const uint32_t d = s_of(r, (uint32_t)l << 3);
                if (d > 255) throw std::runtime_error("delta_r(l) outside F~_{2^8}");
                w |= (uint32_t)H.mul8[(d << 8) | x] << (8 * (r + 1));
            }
            h->low_lane[x][l] = w;
        }
    // phi tables for the shuffle form of changeRepr (phi is F_2-linear)
    for (int q = 0; q < 2; q++)
        for (int w = 0; w < 7; w++)
            for (int l = 0; l < 32; l++) {
                const uint32_t word = w < 6 ? (uint32_t)l << (5 * w) : (uint32_t)(l & 3) << 30;
                u128 acc{0, 0};
                for (int b = 0; b < 4; b++) {
                    const u128 &t = H.chr_in[4 * q + b][(word >> (8 * b)) & 255];
                    acc.lo ^= t.lo;
                    acc.hi ^= t.hi;
                }
                const uint32_t o4[4] = {(uint32_t)acc.lo, (uint32_t)(acc.lo >> 32), (uint32_t)acc.hi,
                                        (uint32_t)(acc.hi >> 32)};
                for (int o = 0; o < 4; o++) h->phi_shfl[o][q][w][l] = o4[o];
            }
    // psi tables for the shuffle form of changeRepr^-1 (psi is F_2-linear)
    for (int q = 0; q < 4; q++)
        for (int w = 0; w < 7; w++)
            for (int l = 0; l < 32; l++) {
                const uint32_t word = w < 6 ? (uint32_t)l << (5 * w) : (uint32_t)(l & 3) << 30;
                u128 acc{0, 0};
                for (int b = 0; b < 4; b++) {
                    const u128 &t = H.chr_out[4 * q + b][(word >> (8 * b)) & 255];
                    acc.lo ^= t.lo;
                    acc.hi ^= t.hi;
                }
                const uint32_t o4[4] = {(uint32_t)acc.lo, (uint32_t)(acc.lo >> 32), (uint32_t)acc.hi,
                                        (uint32_t)(acc.hi >> 32)};
                for (int o = 0; o < 4; o++) h->psi_shfl[o][q][w][l] = o4[o];
            }
    for (int r = 0; r < 3; r++)
        for (int blk = 0; blk < 16; blk++)
            for (int hh = 0; hh < (4 >> r); hh++) {
                uint32_t t[7][32];
                shfl_table_of(s_of(r, ((uint32_t)blk << 8) | ((uint32_t)hh << (r + 1))), t);
                std::memcpy(h->low_shfl[kLowOff[r] + blk * (4 >> r) + hh], t, sizeof(t));
            }
}

void shape_of(uint64_t na_bits, uint64_t nb_bits, int *M, int *pa_log, int *pb_log) {
    const uint64_t na_w = words_of(na_bits), nb_w = words_of(nb_bits);
    *M = log2_ceil(std::max<uint64_t>(2, na_w + nb_w - 1));
    *pa_log = log2_ceil(na_w);
    *pb_log = log2_ceil(nb_w);
}

int plan_init(gf2x_plan *p, uint64_t na_bits, uint64_t nb_bits, PassTableFn src,
              const PlanTune &tune) {
    p->tune = tune;
    p->na_bits = na_bits;
    p->nb_bits = nb_bits;
    p->na_w = words_of(na_bits);
    p->nb_w = words_of(nb_bits);
    p->total_bits = na_bits + nb_bits - 1;
    p->out_words = words_of(p->total_bits);
    // N: the smallest power of two >= na_w + nb_w - 1 (the product's number
    // of 64-bit blocks), so that interpolation at N points is exact.
    const uint64_t need = std::max<uint64_t>(2, p->na_w + p->nb_w - 1);
    p->M = log2_ceil(need);
    if (p->M > kMaxLogN) return -1;
    p->N = 1ull << p->M;
    p->pa_log = log2_ceil(p->na_w);
    p->pb_log = log2_ceil(p->nb_w);
    p->Pa = 1ull << p->pa_log;
    p->Pb = 1ull << p->pb_log;
    p->lv_a = basis_cvt_levels(p->pa_log);
    p->lv_b = basis_cvt_levels(p->pb_log);
    p->lv_c = basis_cvt_levels(p->M);
    int rc = plan_fft_forward(p->M, p->pa_log, p->fft_a, src, tune.fft_depth, tune.fft_nbuf);
    if (rc) return rc;
    if ((rc = plan_fft_fused(p->M, p->pb_log, p->fft_b, p->fused, p->ifft_top, src,
                             tune.fft_depth, tune.fft_nbuf)))
        return rc;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    p->off_fa = 0;
    p->off_fb = up(p->off_fa + 16 * p->N);
    p->off_wa = up(p->off_fb + 16 * p->N);
    p->off_wb = up(p->off_wa + 8 * p->Pa);
    p->off_st = up(p->off_wb + 8 * p->Pb);
    // fft_a ends with its bottom pass; fft_b holds strided passes only
    const bool staged = p->fft_a.n > 1 || p->fft_b.n > 0;
    p->ws_bytes = up(p->off_st + (staged ? 16 * std::max(p->Pa, p->Pb) : 0));
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        return -3;
    }
    return 0;
}

int plan_run_batch(const gf2x_plan *p, int count, const OperandDesc *many_a,
                   const OperandDesc *many_b, const OutputDesc *many_out, const OperandDesc &one_a,
                   const OperandDesc &one_b, const OutputDesc &one_out, uint64_t max_out_words,
                   void *ws, size_t ws_stride, cudaStream_t s, const DevTables *T, int *st,
                   StageHook *hook, cudaEvent_t b_ready, const OutputDrain *drain) {
    char *base = static_cast<char *>(ws);
    uint4 *FA = reinterpret_cast<uint4 *>(base + p->off_fa);
    uint4 *FB = reinterpret_cast<uint4 *>(base + p->off_fb);
    uint64_t *WA = reinterpret_cast<uint64_t *>(base + p->off_wa);
    uint64_t *WB = reinterpret_cast<uint64_t *>(base + p->off_wb);
    uint4 *ST = reinterpret_cast<uint4 *>(base + p->off_st);
    const uint64_t sF = ws_stride / 16, sW = ws_stride / 8;
    auto begin = [&](int stage) {
        if (hook) hook->begin(stage);
    };
    auto end = [&](uint64_t n) {
        if (hook) hook->end(n);
    };
    // Split, BasisCvt, changeRepr + FFT_LCH of a (the layers above log2 Pa
    // are fan-outs: the first pass reads the P converted blocks periodically)
    begin(ST_SPLIT);
    launch_split_pad(one_a, many_a, count, WA, p->Pa, sW, s);
    end(1);
    // with strided passes: changeRepr into ST, which the first pass reads
    // periodically (done by the last BasisCvt tile pass where it is one); a
    // lone bottom pass reads the blocks and converts them itself
    const bool st_a = p->fft_a.n > 1;
    const PhiOut phi{ST, sF, T};
    bool phi_done = false;
    begin(ST_BCVT);
    end(run_basis_cvt<uint64_t>(WA, p->pa_log, p->lv_a, 0, s, count, sW, p->tune.bcvt,
                                st_a ? &phi : nullptr, &phi_done));
    if (st_a && !phi_done) {
        begin(ST_CHREPR);
        launch_chrepr_stage(WA, p->Pa, sW, ST, sF, count, T, s);
        end(1);
    }
    begin(ST_FFT_A);
    for (int i = 0; i < p->fft_a.n; i++)
        launch_fft_pass(p->fft_a.v[i], p->M, FA, (i == 0 && !st_a) ? WA : nullptr, p->Pa, nullptr, T,
                        st, s, count, sF, sW, (i == 0 && st_a) ? ST : nullptr);
    end(p->fft_a.n);
    // the same for b, then its top FFT layers
    if (b_ready) cudaStreamWaitEvent(s, b_ready, 0);
    begin(ST_SPLIT);
    launch_split_pad(one_b, many_b, count, WB, p->Pb, sW, s);
    end(1);
    begin(ST_BCVT);
    end(run_basis_cvt<uint64_t>(WB, p->pb_log, p->lv_b, 0, s, count, sW, p->tune.bcvt,
                                p->fft_b.n > 0 ? &phi : nullptr, &phi_done));
    if (p->fft_b.n > 0 && !phi_done) {
        begin(ST_CHREPR);
        launch_chrepr_stage(WB, p->Pb, sW, ST, sF, count, T, s);
        end(1);
    }
    begin(ST_FFT_B);
    for (int i = 0; i < p->fft_b.n; i++)
        launch_fft_pass(p->fft_b.v[i], p->M, FB, nullptr, p->Pb, nullptr, T, st, s, count, sF, sW,
                        i == 0 ? ST : nullptr);
    end(p->fft_b.n);
    // bottom layers of FFT(b), pointmul, bottom layers of iFFT_LCH
    begin(ST_FUSED);
    launch_fft_pass(p->fused, p->M, FB, p->fft_b.n == 0 ? WB : nullptr, p->Pb, FA, T, st, s, count,
                    sF, sW);
    end(1);
    // iFFT_LCH top layers
    begin(ST_IFFT);
    for (int i = 0; i < p->ifft_top.n; i++)
        launch_fft_pass(p->ifft_top.v[i], p->M, FB, nullptr, 0, nullptr, T, st, s, count, sF, sW);
    end(p->ifft_top.n);
    // iBasisCvt
    begin(ST_IBCVT);
    end(run_basis_cvt<uint4>(FB, p->M, p->lv_c, 1, s, count, sF, p->tune.bcvt));
    // changeRepr^-1 + InterleavedCombine
    begin(ST_OUT);
    if (drain && count == 1 && !many_out && drain->chunks > 1) {
        const uint64_t words = one_out.words, piece = (words + drain->chunks - 1) / drain->chunks;
        for (int c = 0; c < drain->chunks; c++) {
            const uint64_t j0 = std::min(words, c * piece), j1 = std::min(words, j0 + piece);
            launch_ichrepr_combine(FB, p->N, sF, one_out, nullptr, 1, words, T, s, j0, j1);
            cudaEventRecord(drain->events[c], s);
            cudaStreamWaitEvent(drain->stream, drain->events[c], 0);
            if (j1 > j0)
                cudaMemcpyAsync(drain->host + j0, one_out.out + j0, (j1 - j0) * 8,
                                cudaMemcpyDeviceToHost, drain->stream);
        }
        end(drain->chunks);
    } else {
        launch_ichrepr_combine(FB, p->N, sF, one_out, many_out, count,
                               many_out ? max_out_words : one_out.words, T, s);
        end(1);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : -3;
}

uint64_t mask_of_bits(uint64_t bits) { return (bits % 64) ? ((1ull << (bits % 64)) - 1) : ~0ull; }

bool chunk_shape(uint64_t xw, uint64_t yw, ChunkShape *cs) {
    if (yw == 0 || xw < yw) return false;
    // at most 2^15 chunks (one launch row per chunk)
    const uint64_t L = 1ull << std::max(log2_ceil(std::max<uint64_t>(yw, 512)),
                                        log2_ceil((xw + 32767) / 32768));
    const uint64_t C = (xw + L - 1) / L;
    if (C < 4) return false;
    cs->L = L;
    cs->C = C;
    return true;
}

// C chunk workspaces of the chunk plan (chunk i's FB, WB, ST at + i * ws_bytes;
// block 0's FA, WA also hold y's transform), then the descriptors.
size_t chunked_ws_bytes(const gf2x_plan *pc, uint64_t C) {
    const size_t descs = C * (sizeof(OperandDesc) + sizeof(OutputDesc));
    return C * pc->ws_bytes + ((descs + 255) & ~size_t(255));
}

int plan_run_chunked(const gf2x_plan *pc, const ChunkShape &cs, const uint64_t *x,
                     uint64_t x_bits, const uint64_t *y, uint64_t y_bits, uint64_t *out, void *ws,
                     cudaStream_t s, const DevTables *T, int *st, StageHook *hook) {
    const uint64_t C = cs.C, L = cs.L, xw = words_of(x_bits);
    if (C > (uint64_t)INT32_MAX / 2) return -1;
    const int count = (int)C;
    char *base = static_cast<char *>(ws);
    const size_t blk = pc->ws_bytes;
    uint4 *FA = reinterpret_cast<uint4 *>(base + pc->off_fa);
    uint4 *FB = reinterpret_cast<uint4 *>(base + pc->off_fb);
    uint64_t *WA = reinterpret_cast<uint64_t *>(base + pc->off_wa);
    uint64_t *WB = reinterpret_cast<uint64_t *>(base + pc->off_wb);
    uint4 *ST = reinterpret_cast<uint4 *>(base + pc->off_st);
    OperandDesc *dx = reinterpret_cast<OperandDesc *>(base + C * blk);
    OutputDesc *dout = reinterpret_cast<OutputDesc *>(dx + C);
    const uint64_t sF = blk / 16, sW = blk / 8;
    const uint64_t out_words = words_of(x_bits + y_bits - 1);
    auto begin = [&](int stage) {
        if (hook) hook->begin(stage);
    };
    auto end = [&](uint64_t n) {
        if (hook) hook->end(n);
    };
    // y: Split, BasisCvt, changeRepr and every forward layer, once
    const OperandDesc one_y{y, words_of(y_bits), mask_of_bits(y_bits)};
    begin(ST_SPLIT);
    launch_split_pad(one_y, nullptr, 1, WA, pc->Pa, sW, s);
    launch_chunk_descs(x, xw, mask_of_bits(x_bits), L, C, out, out_words,
                       mask_of_bits(x_bits + y_bits - 1), pc->out_words, dx, dout, s);
    end(2);
    begin(ST_BCVT);
    end(run_basis_cvt<uint64_t>(WA, pc->pa_log, pc->lv_a, 0, s, 1, sW, pc->tune.bcvt));
    const bool st_a = pc->fft_a.n > 1;
    if (st_a) {
        begin(ST_CHREPR);
        launch_chrepr_stage(WA, pc->Pa, sW, ST, sF, 1, T, s);
        end(1);
    }
    begin(ST_FFT_A);
    for (int i = 0; i < pc->fft_a.n; i++)
        launch_fft_pass(pc->fft_a.v[i], pc->M, FA, (i == 0 && !st_a) ? WA : nullptr, pc->Pa,
                        nullptr, T, st, s, 1, sF, sW, (i == 0 && st_a) ? ST : nullptr);
    end(pc->fft_a.n);
    // the chunks, as operand b of C products sharing y's transform
    const OperandDesc none{nullptr, 0, 0};
    begin(ST_SPLIT);
    launch_split_pad(none, dx, count, WB, pc->Pb, sW, s);
    end(1);
    begin(ST_BCVT);
    end(run_basis_cvt<uint64_t>(WB, pc->pb_log, pc->lv_b, 0, s, count, sW, pc->tune.bcvt));
    if (pc->fft_b.n > 0) {
        begin(ST_CHREPR);
        launch_chrepr_stage(WB, pc->Pb, sW, ST, sF, count, T, s);
        end(1);
    }
    begin(ST_FFT_B);
    for (int i = 0; i < pc->fft_b.n; i++)
        launch_fft_pass(pc->fft_b.v[i], pc->M, FB, nullptr, pc->Pb, nullptr, T, st, s, count, sF,
                        sW, i == 0 ? ST : nullptr);
    end(pc->fft_b.n);
    begin(ST_FUSED);
    launch_fft_pass(pc->fused, pc->M, FB, pc->fft_b.n == 0 ? WB : nullptr, pc->Pb, FA, T, st, s,
                    count, sF, sW, nullptr, 0);
    end(1);
    begin(ST_IFFT);
    for (int i = 0; i < pc->ifft_top.n; i++)
        launch_fft_pass(pc->ifft_top.v[i], pc->M, FB, nullptr, 0, nullptr, T, st, s, count, sF, sW);
    end(pc->ifft_top.n);
    begin(ST_IBCVT);
    end(run_basis_cvt<uint4>(FB, pc->M, pc->lv_c, 1, s, count, sF, pc->tune.bcvt));
    // the chunk products overlap their neighbours (y's words - 1 at most, no
    // more than L): the even chunks, then the odd ones, XORed into a zeroed
    // output
    begin(ST_OUT);
    cudaMemsetAsync(out, 0, 8 * out_words, s);
    const OutputDesc none_out{nullptr, 0, 0};
    const int even = (count + 1) / 2, odd = count / 2;
    launch_ichrepr_combine(FB, pc->N, 2 * sF, none_out, dout, even, pc->out_words, T, s, 0, ~0ull,
                           true);
    if (odd > 0)
        launch_ichrepr_combine(FB + sF, pc->N, 2 * sF, none_out, dout + even, odd, pc->out_words, T,
                               s, 0, ~0ull, true);
    end(odd > 0 ? 2 : 1);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int plan_run_core(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out,
                  void *ws, cudaStream_t s, const DevTables *T, int *st, StageHook *hook,
                  cudaEvent_t b_ready, const OutputDrain *drain) {
    const OperandDesc da{a, p->na_w, mask_of_bits(p->na_bits)};
    const OperandDesc db{b, p->nb_w, mask_of_bits(p->nb_bits)};
    const OutputDesc dout{out, p->out_words, mask_of_bits(p->total_bits)};
    return plan_run_batch(p, 1, nullptr, nullptr, nullptr, da, db, dout, p->out_words, ws,
                          p->ws_bytes, s, T, st, hook, b_ready, drain);
}

}  // namespace gf2x
