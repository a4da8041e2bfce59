// dd_plan.cpp -- host side of libdd: the Eq. 1 delay table, plan creation,
// the per-variant staging tables of the forward kernel, the variant grid and
// the thread-local error state of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <limits>
#include <sstream>

#include "dd_internal.h"

namespace dd {

namespace {
thread_local dd_status tl_status = DD_OK;
thread_local std::string tl_msg;

// Dispersion constant of Eq. 1 in MHz^2 pc^-1 cm^3 s (the paper prints the
// rounded value 4150).
constexpr double kDispersionConst = 4.148808e3;
constexpr int64_t kMaxShift = int64_t(1) << 30;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int64_t floor_to(int64_t x, int64_t m) { return x >= 0 ? x / m * m : -((-x + m - 1) / m) * m; }
}  // namespace

dd_status fail(dd_status s, const std::string &msg) {
    tl_status = s;
    tl_msg = msg;
    return s;
}
dd_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? DD_ERR_NOMEM : DD_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}
dd_status ok() { return DD_OK; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

dd_status replace_fwd_tables(dd_plan_s *p, FwdTables *cur, const FwdTables &next) {
    cudaError_t e = p->launches.wait();  // no launch of this plan still reads *cur
    if (p->launches.captured)
        p->retired.push_back(*cur);  // a captured graph may replay launches that read it
    else
        free_fwd_tables(cur);
    *cur = next;
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the plan's launches");
    return DD_OK;
}

dd_status check_variant_shape(const dd_variant &v) {
    if (!fwd_variant_compiled(v.kind, v.dm_per_thread, v.samples_per_thread))
        return fail(DD_ERR_ARG, "variant (kind, dm_per_thread, samples_per_thread) not compiled");
    if (v.warps_dm < 1 || v.warps_time < 1 || v.warps_dm * v.warps_time > max_trial_warps(v.kind))
        return fail(DD_ERR_ARG,
                    "variant warps_dm * warps_time must be in [1, 8] (kinds 4 and 6: [1, 16])");
    if (v.chans_per_stage != 4 && v.chans_per_stage != 8 && v.chans_per_stage != 16 &&
        v.chans_per_stage != 32)
        return fail(DD_ERR_ARG, "variant chans_per_stage must be 4, 8, 16 or 32");
    if (v.stages < 2 || v.stages > 4) return fail(DD_ERR_ARG, "variant stages must be 2..4");
    return DD_OK;
}

namespace {

// Sub-band (kind 2) tables of one DM tile and one chunk of channels. For a
// group of up to 4 adjacent channels with reference channel r (its last),
// trial d has base delay base(d) = shift[d][r] and relative pattern
// rho_c(d) = shift[d][c] - base(d). Trials sharing a pattern p read the
// weighted partial series P_p[u] = sum_c w_c * x_c[t0 + u + rho_c], u in
// [Bmin_p, Bmax_p + Ts), at index u = t + base(d); the CTA builds each P_p
// once in shared memory and every trial of p adds one P_p value per output
// instead of one input value per channel.
struct SbChunk {
    std::vector<int> bdesc;   // [groups][kSbPatterns][8]
    std::vector<int> poffs;   // [groups][Dt]
    int64_t p_elems = 0;
};

dd_status sb_chunk(const dd_plan_s *p, int d0, int d1, int Dt, int Ts, int c0, int nch_chunk,
                   const std::vector<int4> &raw_desc_k, SbChunk *out) {
    const int ngroups = (nch_chunk + kSbGroup - 1) / kSbGroup;
    out->bdesc.assign(size_t(ngroups) * kSbPatterns * 8, 0);
    out->poffs.assign(size_t(ngroups) * Dt, 0);
    int64_t psoff = 0;
    for (int g = 0; g < ngroups; ++g) {
        const int ga = c0 + g * kSbGroup;
        const int gn = std::min(kSbGroup, p->C - ga);
        if (gn <= 0) continue;
        const int ref = ga + gn - 1;
        std::vector<std::vector<int32_t>> pats;
        std::vector<int32_t> bmin, bmax;
        std::vector<int> pid(size_t(Dt), 0);
        for (int d = d0; d < d1; ++d) {
            const int32_t base = p->shifts[size_t(d) * p->C + ref];
            std::vector<int32_t> rho(static_cast<size_t>(gn), 0);
            for (int j = 0; j < gn; ++j) rho[size_t(j)] = p->shifts[size_t(d) * p->C + ga + j] - base;
            size_t q = 0;
            while (q < pats.size() && pats[q] != rho) ++q;
            if (q == pats.size()) {
                if (int(q) == kSbPatterns) return DD_ERR_ARG;  // too many patterns for this tile
                pats.push_back(rho);
                bmin.push_back(base);
                bmax.push_back(base);
            }
            bmin[q] = std::min(bmin[q], base);
            bmax[q] = std::max(bmax[q], base);
            pid[size_t(d - d0)] = int(q);
        }
        std::vector<int64_t> pso(pats.size());
        for (size_t q = 0; q < pats.size(); ++q) {
            // each series takes a whole number of 32-element build blocks
            const int64_t L = int64_t(bmax[q]) - bmin[q] + Ts;
            pso[q] = psoff;
            int *bd = &out->bdesc[(size_t(g) * kSbPatterns + q) * 8];
            bd[0] = int(psoff);
            bd[1] = int(L);
            for (int j = 0; j < gn; ++j) {
                const int4 r = raw_desc_k[size_t(ga + j)];  // {ws, len, soff, 0}
                bd[2 + j] = int(r.z + bmin[q] + pats[q][size_t(j)] - r.x);
            }
            bd[6] = gn;
            psoff += round_up(L, 32);
        }
        for (int i = 0; i < Dt; ++i) {
            const int d = d0 + i;
            if (d >= d1) continue;
            const int q = pid[size_t(i)];
            out->poffs[size_t(g) * Dt + i] =
                int(pso[size_t(q)] + p->shifts[size_t(d) * p->C + ref] - bmin[size_t(q)]);
        }
    }
    out->p_elems = psoff;
    return DD_OK;
}

}  // namespace

dd_status build_fwd_tables(dd_plan_s *p, const dd_variant &v, FwdTables *out) {
    dd_status s = check_variant_shape(v);
    if (s != DD_OK) return s;
    FwdTables t;
    t.v = v;
    t.Dt = v.dm_per_thread * v.warps_dm;
    t.Ts = 32 * v.samples_per_thread * v.warps_time;
    t.n_dtiles = (p->D + t.Dt - 1) / t.Dt;
    t.n_ttiles = static_cast<int>((p->S + t.Ts - 1) / t.Ts);
    const int cch = v.chans_per_stage;
    t.C_pad = (p->C + cch - 1) / cch * cch;
    const int al = align_elems(p->dtype);
    const int elt = elt_bytes(p->dtype);
    const bool sb = is_subband(v.kind);
    if (int64_t(t.n_ttiles) * t.n_dtiles > 0x7fffffffLL)
        return fail(DD_ERR_ARG, "too many tiles for this variant");
    if (sb && t.Dt % 8 != 0) return fail(DD_ERR_ARG, "sub-band variants need 8 | DM tile");
    if (sb && v.kind != 6 && cch > 16 && p->dtype == DD_F32)
        return fail(DD_ERR_ARG, "sub-band kinds 2-4 with FP32 input stage at most 16 channels");

    const int G_pad = t.C_pad / kSbGroup;
    // desc: each channel's union window {ws, len, soff} per DM tile (the
    // sub-band build reads it); copies: the staging copies of each (DM tile,
    // chunk) {ws, len, soff, channel in the chunk}, laid out with a common
    // capacity once every chunk is known.
    std::vector<int4> desc(size_t(t.n_dtiles) * t.C_pad, make_int4(0, 0, 0, 0));
    std::vector<uint16_t> offs(sb ? size_t(t.n_dtiles) * G_pad * t.Dt
                                  : size_t(t.n_dtiles) * t.C_pad * t.Dt, 0);
    // sub-band build blocks, per (DM tile, chunk); laid out with a common
    // capacity once every chunk is known
    const int n_chunks = (p->C + cch - 1) / cch;
    std::vector<std::vector<int4>> blocks(sb ? size_t(t.n_dtiles) * n_chunks : 0);
    std::vector<std::vector<int4>> copies(size_t(t.n_dtiles) * n_chunks);
    int64_t stage_max = 0, p_max = 0;
    t.dtile_max_shift.assign(size_t(t.n_dtiles), 0);
    std::vector<int32_t> tsh(size_t(t.Dt));
    std::vector<int> order(size_t(t.Dt)), seg_of(size_t(t.Dt));
    std::vector<int64_t> seg_ws, seg_soff;
    for (int k = 0; k < t.n_dtiles; ++k) {
        const int d0 = k * t.Dt, d1 = std::min(p->D, d0 + t.Dt);
        const int nd = d1 - d0;
        for (int c0 = 0; c0 < p->C; c0 += cch) {
            int64_t soff = 0;
            std::vector<int4> &cl = copies[size_t(k) * n_chunks + c0 / cch];
            for (int c = c0; c < std::min(p->C, c0 + cch); ++c) {
                int32_t smin = std::numeric_limits<int32_t>::max(), smax = 0;
                for (int i = 0; i < nd; ++i) {
                    tsh[size_t(i)] = p->shifts[size_t(d0 + i) * p->C + c];
                    smin = std::min(smin, tsh[size_t(i)]);
                    smax = std::max(smax, tsh[size_t(i)]);
                }
                t.dtile_max_shift[size_t(k)] = std::max(t.dtile_max_shift[size_t(k)], smax);
                {
                    const int64_t ws = floor_to(smin, al);
                    desc[size_t(k) * t.C_pad + c] =
                        make_int4(int(ws), int(round_up(smax + t.Ts - ws, al)), int(soff), 0);
                }
                // Windows [shift, shift + Ts) of the tile's trials, in delay
                // order, are merged while they overlap or touch; the
                // sub-band kinds take the whole union as one window. A
                // channel whose delay steps by more than a time tile between
                // trials (low frequencies, coarse DM grids, fine sampling)
                // thus stages one window per trial instead of a union that
                // is mostly gaps.
                for (int i = 0; i < nd; ++i) order[size_t(i)] = i;
                std::sort(order.begin(), order.begin() + nd,
                          [&](int x, int y) { return tsh[size_t(x)] < tsh[size_t(y)]; });
                seg_ws.clear();
                seg_soff.clear();
                int64_t lo = tsh[size_t(order[0])], hi = lo;
                auto close_seg = [&]() -> bool {
                    const int64_t ws = floor_to(lo, al);
                    const int64_t len = round_up(hi + t.Ts - ws, al);
                    if (soff + len > 65536) return false;
                    cl.push_back(make_int4(int(ws), int(len), int(soff), c - c0));
                    seg_ws.push_back(ws);
                    seg_soff.push_back(soff);
                    soff += len;
                    return true;
                };
                for (int r = 0; r < nd; ++r) {
                    const int i = order[size_t(r)];
                    const int64_t sh = tsh[size_t(i)];
                    if (!sb && sh > hi + t.Ts) {
                        if (!close_seg()) return fail(DD_ERR_ARG, "stage too large for variant");
                        lo = sh;
                    }
                    hi = std::max<int64_t>(hi, sh);
                    seg_of[size_t(i)] = int(seg_ws.size());
                }
                if (!close_seg()) return fail(DD_ERR_ARG, "stage too large for variant");
                if (!sb) {
                    for (int i = 0; i < t.Dt; ++i) {
                        int64_t o = seg_soff[0];  // trials beyond D: any in-range offset
                        if (i < nd) {
                            const size_t q = size_t(seg_of[size_t(i)]);
                            o = seg_soff[q] + tsh[size_t(i)] - seg_ws[q];
                        }
                        offs[(size_t(k) * t.C_pad + c) * t.Dt + i] = static_cast<uint16_t>(o);
                    }
                }
            }
            stage_max = std::max(stage_max, soff);
            if (sb) {
                SbChunk ch;
                std::vector<int4> raw_k(desc.begin() + size_t(k) * t.C_pad,
                                        desc.begin() + size_t(k + 1) * t.C_pad);
                if (sb_chunk(p, d0, d1, t.Dt, t.Ts, c0, std::min(cch, p->C - c0), raw_k, &ch) !=
                    DD_OK)
                    return fail(DD_ERR_ARG, "too many delay patterns per channel group");
                if (ch.p_elems > 65536 - t.Ts)
                    return fail(DD_ERR_ARG, "partial-sum buffer too large for variant");
                p_max = std::max(p_max, ch.p_elems);
                const int g0 = c0 / kSbGroup;
                const int ng = int(ch.poffs.size()) / t.Dt;
                // Build blocks: every partial series is cut into blocks of up
                // to 4 x 32 elements, {dst, r0, (r1-r0) | (r2-r0) << 16, (r3-r0)
                // | group << 16 | channels << 20 | sub-blocks << 24} with the
                // relative offsets as int16 (lane l of sub-block s builds
                // dst[32 s + l] = sum_j w_j raw[r_j + 32 s + l]); the series'
                // buffer lengths are whole 32-element sub-blocks, so no lane
                // writes past its series.
                std::vector<int4> &bl = blocks[size_t(k) * n_chunks + c0 / cch];
                for (int g = 0; g < ng; ++g) {
                    for (int i = 0; i < t.Dt; ++i)
                        offs[(size_t(k) * G_pad + g0 + g) * t.Dt + i] =
                            static_cast<uint16_t>(ch.poffs[size_t(g) * t.Dt + i]);
                    for (int q = 0; q < kSbPatterns; ++q) {
                        const int *bd = &ch.bdesc[(size_t(g) * kSbPatterns + q) * 8];
                        if (bd[1] == 0) continue;
                        const int gn = bd[6];
                        int rel[4] = {0, 0, 0, 0};
                        for (int j = 1; j < gn; ++j) {
                            rel[j] = bd[2 + j] - bd[2];
                            if (rel[j] < -32768 || rel[j] > 32767)
                                return fail(DD_ERR_ARG, "channel windows too far apart for variant");
                        }
                        for (int u = 0; u < bd[1]; u += 128) {
                            const int nsub = std::min(4, (bd[1] - u + 31) / 32);
                            bl.push_back(make_int4(
                                bd[0] + u, bd[2] + u,
                                int((uint32_t(rel[1]) & 0xffffu) | (uint32_t(rel[2]) << 16)),
                                int((uint32_t(rel[3]) & 0xffffu) | (uint32_t(g) << 16) |
                                    (uint32_t(gn) << 20) | (uint32_t(nsub) << 24))));
                        }
                    }
                }
            }
        }
    }
    // staging copies with a common capacity (length-0 entries pad); one warp
    // issues a chunk's copies, one per lane
    t.n_copies = 1;
    for (const auto &cl : copies) t.n_copies = std::max<int>(t.n_copies, int(cl.size()));
    if (t.n_copies > 32)
        return fail(DD_ERR_ARG, "more than 32 staging windows per chunk for this variant");
    std::vector<int4> copy_tab(copies.size() * size_t(t.n_copies), make_int4(0, 0, 0, 0));
    for (size_t i = 0; i < copies.size(); ++i)
        std::copy(copies[i].begin(), copies[i].end(), copy_tab.begin() + i * size_t(t.n_copies));
    std::vector<int4> bdesc;
    if (sb) {
        // Worker w of `parts` builds blocks w, w + parts, ... of a chunk in
        // this order (series by series). (Assigning blocks longest first to
        // the least-loaded worker measured slower on GB300.)
        size_t cap = 1;
        for (const auto &bl : blocks) cap = std::max(cap, bl.size());
        t.n_blocks = int(cap);
        bdesc.assign(blocks.size() * cap, make_int4(0, 0, 0, 0));  // 0 sub-blocks: no block
        for (size_t i = 0; i < blocks.size(); ++i)
            std::copy(blocks[i].begin(), blocks[i].end(), bdesc.begin() + i * cap);
    }
    t.stage_elems = static_cast<int>(stage_max);
    // 64 spare elements: register-window loads of a warp and the last lanes of
    // a build block never leave the slot
    t.stage_data_bytes = static_cast<int>(round_up((stage_max + 64) * elt, 16));
    // per slot after the window data: the chunk's tables, then its weights
    if (sb) {
        const int gpc = cch / kSbGroup;
        t.stage_offs_bytes = static_cast<int>(round_up(int64_t(gpc) * t.Dt * 2, 16)) +
                             t.n_blocks * 16 + cch * 4;
        t.p_elems = static_cast<int>(round_up(p_max + 64, 4));
    } else {
        t.stage_offs_bytes = static_cast<int>(round_up(int64_t(cch) * t.Dt * 2, 16)) + cch * 4;
    }
    size_t p_bytes = 0;
    if (v.kind == 2 || v.kind == 4)  // 2 partial-sum slots, each with the chunk's trial offsets
        p_bytes = size_t(2) * (size_t(t.p_elems) * 4 + size_t(cch / kSbGroup) * t.Dt * 2);
    if (v.kind == 6)  // 1 partial-sum slot
        p_bytes = size_t(t.p_elems) * 4 + size_t(cch / kSbGroup) * t.Dt * 2;
    if (v.kind == 3)  // 3 partial-sum slots, each with the chunk's trial offsets
        p_bytes = size_t(3) * (size_t(t.p_elems) * 4 + size_t(cch / kSbGroup) * t.Dt * 2);
    t.smem_bytes = 128 + size_t(v.stages) * (t.stage_data_bytes + t.stage_offs_bytes) + p_bytes;
    if (t.smem_bytes > p->smem_optin)
        return fail(DD_ERR_ARG, "variant needs more shared memory than the device has");

    // Live chunk ranges (plans whose input is zero outside [nz_lo, nz_hi) of
    // each row): chunk j of DM tile k can add a nonzero term in time tile tt
    // only if one of its channels' windows [t0 + ws, t0 + ws + len) meets the
    // nonzero columns; per (k, tt) the hull of those chunks is kept.
    std::vector<int2> live;
    if (p->nz_hi >= 0) {
        live.assign(size_t(t.n_dtiles) * t.n_ttiles, make_int2(0, 0));
        for (int k = 0; k < t.n_dtiles; ++k)
            for (int tt = 0; tt < t.n_ttiles; ++tt) {
                const int64_t t0 = int64_t(tt) * t.Ts;
                int first = -1, last = -1;
                for (int j = 0; j < n_chunks; ++j) {
                    bool any = false;
                    for (const int4 &d : copies[size_t(k) * n_chunks + j])
                        any = any || (t0 + d.x < p->nz_hi && t0 + d.x + d.y > p->nz_lo);
                    if (any) {
                        if (first < 0) first = j;
                        last = j;
                    }
                }
                if (first >= 0) live[size_t(k) * t.n_ttiles + tt] = make_int2(first, last + 1);
            }
    }

    // Stream-ordered allocation and upload on the plan's own stream, which
    // is then synchronised (only it): the tables are complete before any
    // launch on another stream can read them, and freeing them later needs
    // no device-wide synchronisation.
    t.aux = p->aux;
    auto upload = [&](void **dst, const void *src, size_t bytes) {
        cudaError_t r = cudaMallocAsync(dst, bytes, t.aux);
        if (r == cudaSuccess) r = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, t.aux);
        return r;
    };
    cudaError_t e = upload(reinterpret_cast<void **>(&t.d_copies), copy_tab.data(),
                           copy_tab.size() * sizeof(int4));
    if (e == cudaSuccess && !live.empty())
        e = upload(reinterpret_cast<void **>(&t.d_live), live.data(), live.size() * sizeof(int2));
    if (e == cudaSuccess)
        e = upload(reinterpret_cast<void **>(&t.d_offs), offs.data(), offs.size() * sizeof(uint16_t));
    if (e == cudaSuccess && sb)
        e = upload(reinterpret_cast<void **>(&t.d_bdesc), bdesc.data(), bdesc.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaStreamSynchronize(t.aux);
    if (e != cudaSuccess) {
        free_fwd_tables(&t);
        return cuda_fail(e, "uploading the staging tables");
    }
    *out = t;
    return DD_OK;
}

// Stream-ordered free on the stream the tables were allocated on; callers
// make sure no launch still reads them (LaunchTracker::wait, or their own
// synchronisation).
void free_fwd_tables(FwdTables *t) {
    void *ptrs[] = {t->d_copies, t->d_offs, t->d_bdesc, t->d_live};
    for (void *q : ptrs)
        if (q) cudaFreeAsync(q, t->aux);
    t->d_copies = nullptr;
    t->d_offs = nullptr;
    t->d_bdesc = nullptr;
    t->d_live = nullptr;
}

namespace {

// Candidate default variants, best first; the first that fits the plan is
// used until dd_tune or dd_plan_set_variant picks another.
// (Measured on GB300: the wide sub-band kinds with 64-trial by 256-sample
// tiles lead on the Apertif-like and 512-channel setups, kind 6 with 32
// channels per stage first (2.34 against 2.43 ms for kind 4 with 16 at the
// survey scale), then kind 2's 64 x 128 tiles; the lane-strided kind 0
// takes setups whose delay patterns are too varied for sub-bands, e.g.
// wide low-frequency bands.)
const dd_variant kDefaults[] = {
    {6, 4, 8, 16, 1, 32, 2}, {4, 4, 8, 16, 1, 16, 2}, {2, 8, 4, 8, 1, 16, 2}, {2, 8, 4, 4, 2, 8, 2},
    {0, 4, 8, 4, 1, 8, 3},   {0, 4, 4, 4, 2, 8, 3},  {0, 4, 4, 4, 2, 4, 2},
    {0, 2, 4, 4, 2, 4, 2},   {0, 4, 2, 4, 1, 4, 2},
};

}  // namespace

// ---- tuning cache: lines "<key> kind dpt spt warps_dm warps_time cch stages"
// in the file named by DD_TUNE_CACHE; the key is the device name, input type,
// shape and a hash of the delay table, so a tuned variant is reused only for
// the same problem on the same kind of GPU.
std::string plan_signature(const dd_plan_s *p) {
    cudaDeviceProp prop{};
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) dev = prop.name;
    for (char &ch : dev)
        if (ch == ' ') ch = '_';
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the delay table
    for (int32_t v : p->shifts) {
        for (int i = 0; i < 4; ++i) {
            h ^= uint64_t((uint32_t(v) >> (8 * i)) & 0xffu);
            h *= 1099511628211ull;
        }
    }
    std::ostringstream os;
    os << dev << "/t" << int(p->dtype) << "/C" << p->C << "/D" << p->D << "/S" << p->S << "/B"
       << p->B << "/" << std::hex << h;
    return os.str();
}

// Lines "<key> kind dpt spt warps_dm warps_time cch stages [time_major]"; a
// line without the last field (written before the launch order was tuned)
// means DM tiles fastest.
bool cache_lookup(const std::string &key, dd_variant *v, bool *time_major) {
    const char *path = std::getenv("DD_TUNE_CACHE");
    if (!path || !*path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {  // the last entry for a key wins
        std::istringstream is(line);
        std::string k;
        dd_variant t{};
        if (is >> k >> t.kind >> t.dm_per_thread >> t.samples_per_thread >> t.warps_dm >>
            t.warps_time >> t.chans_per_stage >> t.stages) {
            int tm = 0;
            if (!(is >> tm)) tm = 0;
            if (k == key) {
                *v = t;
                *time_major = tm != 0;
                found = true;
            }
        }
    }
    return found;
}

void cache_store(const std::string &key, const dd_variant &v, bool time_major) {
    const char *path = std::getenv("DD_TUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream f(path, std::ios::app);
    f << key << " " << v.kind << " " << v.dm_per_thread << " " << v.samples_per_thread << " "
      << v.warps_dm << " " << v.warps_time << " " << v.chans_per_stage << " " << v.stages << " "
      << (time_major ? 1 : 0) << "\n";
}

namespace {

dd_status finish_plan(dd_plan_s *p, dd_plan *out) {
    p->max_shift = 0;
    for (int32_t s : p->shifts) p->max_shift = std::max(p->max_shift, s);
    p->T_in = p->S + p->max_shift;
    p->stride = round_up(p->T_in, align_elems(p->dtype));

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SMs)");
    p->sm_count = v;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(smem)");
    p->smem_optin = size_t(v);
    e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate(plan)");
    e = cudaMalloc(&p->d_shifts, p->shifts.size() * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(shifts)");
    e = cudaMemcpy(p->d_shifts, p->shifts.data(), p->shifts.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(shifts)");
    e = cudaMalloc(&p->d_err, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(err)");
    e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(err)");

    dd_status s = DD_ERR_UNSUPPORTED;
    // 8- and 16-bit input: the wide sub-band CTAs fit 32 channels per stage
    // (a quarter or half of the FP32 staging bytes), which halves the chunk
    // barriers (measured on GB300 at the survey scale: 2.26 against 2.61 ms
    // with 16 channels per stage for 8-bit input)
    const dd_variant narrow_default = {4, 4, 8, 16, 1, 32, 2};
    dd_variant cached{};
    bool cached_tm = false;
    if (cache_lookup(plan_signature(p), &cached, &cached_tm)) {
        s = build_fwd_tables(p, cached, &p->fwd);
        if (s == DD_OK) p->fwd.time_major = cached_tm;
    }
    if (s != DD_OK && p->dtype != DD_F32) {
        s = build_fwd_tables(p, narrow_default, &p->fwd);
        if (s != DD_OK && s != DD_ERR_ARG) return s;
    }
    for (size_t i = 0; s != DD_OK && i < sizeof(kDefaults) / sizeof(kDefaults[0]); ++i) {
        s = build_fwd_tables(p, kDefaults[i], &p->fwd);
        if (s != DD_OK && s != DD_ERR_ARG) return s;
    }
    if (s != DD_OK)
        return fail(DD_ERR_UNSUPPORTED, "no forward variant fits this plan (delay spans too wide)");
    *out = p;
    return ok();
}

dd_status check_common(dd_plan *out, int32_t n_chan, int32_t n_dm, int64_t n_out,
                       int32_t batch, dd_dtype t) {
    if (!out) return fail(DD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_chan < 1 || n_dm < 1 || n_out < 1 || batch < 1)
        return fail(DD_ERR_ARG, "n_chan, n_dm, n_out and batch must be >= 1");
    if (t != DD_F32 && t != DD_F16 && t != DD_BF16 && t != DD_U8)
        return fail(DD_ERR_ARG, "unknown input dtype");
    if (n_out > (int64_t(1) << 31) - (int64_t(1) << 30) || batch > 65535)
        return fail(DD_ERR_ARG, "n_out or batch too large");
    return DD_OK;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_compute_shifts(int32_t n_chan, const double *freq_mhz, double f_ref_mhz,
                            double t_samp_s, int32_t n_dm, const double *dm,
                            int32_t *shifts) {
    if (!freq_mhz || !dm || !shifts) return fail(DD_ERR_ARG, "null pointer");
    if (n_chan < 1 || n_dm < 1) return fail(DD_ERR_ARG, "n_chan and n_dm must be >= 1");
    if (!(t_samp_s > 0.0) || !std::isfinite(t_samp_s))
        return fail(DD_ERR_ARG, "t_samp must be positive and finite");
    if (!(f_ref_mhz > 0.0) || !std::isfinite(f_ref_mhz))
        return fail(DD_ERR_ARG, "f_ref must be positive and finite");
    for (int32_t c = 0; c < n_chan; ++c)
        if (!(freq_mhz[c] > 0.0) || !std::isfinite(freq_mhz[c]))
            return fail(DD_ERR_ARG, "channel frequencies must be positive and finite");
    for (int32_t d = 0; d < n_dm; ++d)
        if (!std::isfinite(dm[d])) return fail(DD_ERR_ARG, "DM values must be finite");
    const double ref_term = 1.0 / (f_ref_mhz * f_ref_mhz);
    for (int32_t d = 0; d < n_dm; ++d) {
        const double k_dm = kDispersionConst * dm[d];
        for (int32_t c = 0; c < n_chan; ++c) {
            const double f = freq_mhz[c];
            const double delay_s = k_dm * (1.0 / (f * f) - ref_term);
            const double r = std::llround(delay_s / t_samp_s);
            if (r < 0) return fail(DD_ERR_ARG, "negative delay: channel above f_ref or DM < 0");
            if (r > double(kMaxShift)) return fail(DD_ERR_ARG, "delay exceeds 2^30 samples");
            shifts[size_t(d) * n_chan + c] = static_cast<int32_t>(r);
        }
    }
    return DD_OK;
}

dd_status dd_plan_create(dd_plan *out, int32_t n_chan, const double *freq_mhz,
                         double f_ref_mhz, double t_samp_s, int32_t n_dm, const double *dm,
                         int64_t n_out, int32_t batch, dd_dtype in_dtype) {
    dd_status s = check_common(out, n_chan, n_dm, n_out, batch, in_dtype);
    if (s != DD_OK) return s;
    auto *p = new (std::nothrow) dd_plan_s;
    if (!p) return fail(DD_ERR_NOMEM, "host allocation");
    p->C = n_chan;
    p->D = n_dm;
    p->B = batch;
    p->S = n_out;
    p->dtype = in_dtype;
    p->shifts.resize(size_t(n_dm) * n_chan);
    s = dd_compute_shifts(n_chan, freq_mhz, f_ref_mhz, t_samp_s, n_dm, dm, p->shifts.data());
    if (s == DD_OK) s = finish_plan(p, out);
    if (s != DD_OK) dd_plan_destroy(p);
    return s;
}

dd_status dd_plan_create_from_shifts(dd_plan *out, int32_t n_chan, int32_t n_dm,
                                     const int32_t *shifts, int64_t n_out, int32_t batch,
                                     dd_dtype in_dtype) {
    dd_status s = check_common(out, n_chan, n_dm, n_out, batch, in_dtype);
    if (s != DD_OK) return s;
    if (!shifts) return fail(DD_ERR_ARG, "shifts is NULL");
    for (size_t i = 0; i < size_t(n_chan) * n_dm; ++i)
        if (shifts[i] < 0 || shifts[i] > kMaxShift)
            return fail(DD_ERR_ARG, "shifts must lie in [0, 2^30]");
    auto *p = new (std::nothrow) dd_plan_s;
    if (!p) return fail(DD_ERR_NOMEM, "host allocation");
    p->C = n_chan;
    p->D = n_dm;
    p->B = batch;
    p->S = n_out;
    p->dtype = in_dtype;
    p->shifts.assign(shifts, shifts + size_t(n_dm) * n_chan);
    s = finish_plan(p, out);
    if (s != DD_OK) dd_plan_destroy(p);
    return s;
}

void dd_plan_destroy(dd_plan p) {
    if (!p) return;
    p->launches.wait();
    free_fwd_tables(&p->fwd);
    for (FwdTables &t : p->retired) free_fwd_tables(&t);
    if (p->aux) cudaStreamSynchronize(p->aux);
    free_adj_state(&p->adj);
    if (p->d_err) cudaFree(p->d_err);
    if (p->d_shifts) cudaFree(p->d_shifts);
    for (cudaEvent_t &ev : p->hx_event)
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t &xs : p->hx_stream)
        if (xs) cudaStreamDestroy(xs);
    if (p->h_in_dev) cudaFree(p->h_in_dev);
    if (p->h_w_dev) cudaFree(p->h_w_dev);
    if (p->h_out_dev) cudaFree(p->h_out_dev);
    p->launches.destroy();
    if (p->aux) cudaStreamDestroy(p->aux);
    delete p;
}

int64_t dd_plan_input_len(dd_plan p) { return p ? p->T_in : -1; }
int64_t dd_plan_input_stride(dd_plan p) { return p ? p->stride : -1; }
int32_t dd_plan_max_shift(dd_plan p) { return p ? p->max_shift : -1; }

dd_status dd_plan_shifts(dd_plan p, int32_t *host_dst) {
    if (!p || !host_dst) return fail(DD_ERR_ARG, "null argument");
    std::memcpy(host_dst, p->shifts.data(), p->shifts.size() * sizeof(int32_t));
    return DD_OK;
}

dd_status dd_plan_get_variant(dd_plan p, dd_variant *v) {
    if (!p || !v) return fail(DD_ERR_ARG, "null argument");
    *v = p->fwd.v;
    return DD_OK;
}

dd_status dd_plan_set_variant(dd_plan p, const dd_variant *v) {
    if (!p || !v) return fail(DD_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(p->mu);
    FwdTables t;
    dd_status s = build_fwd_tables(p, *v, &t);
    if (s != DD_OK) return s;
    return replace_fwd_tables(p, &p->fwd, t);  // waits for this plan's launches only
}

dd_status dd_plan_get_launch_order(dd_plan p, int32_t *order) {
    if (!p || !order) return fail(DD_ERR_ARG, "null argument");
    *order = p->fwd.time_major ? DD_ORDER_TIME_FASTEST : DD_ORDER_DM_FASTEST;
    return DD_OK;
}

dd_status dd_plan_set_launch_order(dd_plan p, int32_t order) {
    if (!p) return fail(DD_ERR_ARG, "null plan");
    if (order != DD_ORDER_DM_FASTEST && order != DD_ORDER_TIME_FASTEST)
        return fail(DD_ERR_ARG, "launch order must be DD_ORDER_DM_FASTEST or DD_ORDER_TIME_FASTEST");
    std::lock_guard<std::mutex> lk(p->mu);
    p->fwd.time_major = order == DD_ORDER_TIME_FASTEST;  // read at each launch; tables unchanged
    return DD_OK;
}

// The variant grid: every compiled (kind, dm_per_thread, samples_per_thread)
// key with every CTA shape, then chunk size and staging depth innermost.
namespace {
const int kShapes[6][2] = {{4, 2}, {2, 4}, {8, 1}, {1, 8}, {4, 1}, {2, 2}};
const int kCch[4] = {8, 16, 4, 32};
const int kStages[3] = {3, 2, 4};
}  // namespace

int32_t dd_variant_count(void) {
    return int32_t(fwd_compiled_keys().size()) * 6 * kStagingChoices;
}

dd_status dd_variant_get(int32_t i, dd_variant *v) {
    if (!v || i < 0 || i >= dd_variant_count()) return fail(DD_ERR_ARG, "variant index");
    const auto &keys = fwd_compiled_keys();
    const int st = i % 3;
    i /= 3;
    const int cc = i % 4;
    i /= 4;
    const int ws = i % 6;
    i /= 6;
    const FwdKernelKey k = keys[size_t(i)];
    // kind 4 runs twice the trial warps of each shape along DM
    const int wdm = kShapes[ws][0] * ((k.kind == 4 || k.kind == 6) ? 2 : 1);
    *v = dd_variant{k.kind, k.dpt, k.spt, wdm, kShapes[ws][1], kCch[cc], kStages[st]};
    return DD_OK;
}

dd_status dd_plan_check_device(dd_plan p) {
    if (!p) return fail(DD_ERR_ARG, "null plan");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(err)");
    e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(err)");
    if (h & kErrWaitTimeout) return fail(DD_ERR_TIMEOUT, "a kernel gave up a bounded wait");
    if (h) return fail(DD_ERR_DEVICE, "a kernel reported a device-side error");
    return DD_OK;
}

const char *dd_status_str(dd_status s) {
    switch (s) {
        case DD_OK: return "DD_OK";
        case DD_ERR_ARG: return "DD_ERR_ARG";
        case DD_ERR_CUDA: return "DD_ERR_CUDA";
        case DD_ERR_NOMEM: return "DD_ERR_NOMEM";
        case DD_ERR_UNSUPPORTED: return "DD_ERR_UNSUPPORTED";
        case DD_ERR_TIMEOUT: return "DD_ERR_TIMEOUT";
        case DD_ERR_NOT_TUNED: return "DD_ERR_NOT_TUNED";
        case DD_ERR_DEVICE: return "DD_ERR_DEVICE";
    }
    return "DD_ERR_UNKNOWN";
}

dd_status dd_get_last_error(void) { return tl_status; }
const char *dd_last_error_message(void) { return tl_msg.c_str(); }
int32_t dd_version(void) { return DD_VERSION; }

}  // extern "C"
