// plan.cpp -- window search and index maps for the two convolution packings
// of Section 3.3.
//
// Conventional (row-major, the packing the paper builds on; left half of
// Fig. 7): the input is zero-padded to H' x W' and cut into square windows of
// side s (clipped to the padded image) holding C_n channels at stride H_n W_n;
// the kernel is stored reversed at offset O = (C_n-1) H_n W_n + (h-1) W_n + h-1
// and output (a, b) of a window is coefficient O + a W_n + b.
//
// Correlated (Eq. 1 and Eq. 2): per channel x^[i O + j] = x[i, j] and
// w^[(h-1-k) O + (h-1-l)] = w[k, l] with O = max(W_w, H_w) + h - 1 over the
// unpadded window; C_n channels are placed at stride S (kernel channels in
// reverse order) where S is the smallest stride that keeps cross-channel terms
// off the requested outputs; C_n is the largest count for which the requested
// outputs stay below N and no wrapped (x^N = -1) term lands on them.
//
// Output packing: Mn kernels share one polynomial at stride Sout (kernel m at
// offset (m mod Mn) Sout), Sout being the smallest stride that keeps the
// other kernels' products off a kernel's requested outputs and Mn the largest
// count for which every requested output stays below N and no wrapped term
// lands on one.
//
// Window choice: minimise the polynomial products per image MG*G*T, then the
// input polynomials G*T, then G, then prefer the larger window.  The paper's
// objective is printed with floors and W_w + h - 1 in a denominator; this is
// the reading used everywhere in the library.
#include <algorithm>
#include <climits>
#include <cstring>

#include "internal.h"

namespace he {

struct Tile { int a0, a1, b0, b1, r0, r1, s0, s1; };
struct Span { long long rlo, rhi, D; };  // requested range and highest degree of one product

// (Mn, Sout) for the given product spans.  Depthwise layers (output channel m
// reads input channel m only) with several channel groups keep Mn a divisor
// of Cn, so the Mn outputs of a kernel polynomial lie in one channel group and
// every output takes exactly one (kernel polynomial, channel group) product
// (with one group that holds for any Mn).
static void out_packing(int M, long long N, const std::vector<Span> &sp, int &Mn, long long &Sout, int depthwise_cn) {
    Sout = 0;
    for (const Span &e : sp) Sout = std::max(Sout, std::max(e.rhi, e.D - e.rlo));
    Sout += 1;
    auto fits = [&](long long k) {
        for (const Span &e : sp) {
            if ((k - 1) * Sout + e.rhi >= N) return false;
            const long long tot = (k - 1) * Sout + e.D;
            if (!(tot < N || tot - N < e.rlo)) return false;
        }
        return true;
    };
    int k = 1;
    while (k < M && fits(k + 1)) k++;
    if (depthwise_cn > 0) {
        while (depthwise_cn % k) k--;
        Mn = k;
        return;
    }
    const int G = (M + k - 1) / k;
    Mn = (M + G - 1) / G;
}

// products per image: every (kernel polynomial, channel group) pair, or one
// per kernel polynomial for a depthwise layer
static long long plan_products(bool depthwise, long long MG, long long G, long long T) {
    return depthwise ? MG * T : MG * G * T;
}

static bool conv_search(int N, const he_conv_shape &s, bool dw, he_plan_info &I, std::vector<Tile> &tiles) {
    const int Hp = s.H + 2 * s.pad, Wp = s.W + 2 * s.pad;
    const int Ho = Hp - s.h + 1, Wo = Wp - s.h + 1;
    long long best[5] = {LLONG_MAX, 0, 0, 0, 0};
    bool found = false;
    for (int G = 1; G <= s.C; G++) {
        const int Cn = (s.C + G - 1) / G;
        if ((s.C + Cn - 1) / Cn != G) continue;
        for (int side = s.h; side <= std::max(Hp, Wp); side++) {
            const int Hn = std::min(side, Hp), Wn = std::min(side, Wp);
            if ((long long)Cn * Hn * Wn > N) continue;
            const int th = Hn - s.h + 1, tw = Wn - s.h + 1;
            const int Th = (Ho + th - 1) / th, Tw = (Wo + tw - 1) / tw;
            const long long O = (long long)(Cn - 1) * Hn * Wn + (long long)(s.h - 1) * Wn + s.h - 1;
            const long long D = (long long)Cn * Hn * Wn - 1 + O;
            std::vector<Span> sp;
            for (int i = 0; i < Th; i++)
                for (int j = 0; j < Tw; j++) {
                    const int a = std::min(th, Ho - i * th), b = std::min(tw, Wo - j * tw);
                    sp.push_back({O, O + (long long)(a - 1) * Wn + (b - 1), D});
                }
            int Mn;
            long long Sout;
            out_packing(s.M, N, sp, Mn, Sout, dw && G > 1 ? Cn : 0);
            const long long MG = (s.M + Mn - 1) / Mn;
            long long key[5] = {plan_products(dw, MG, G, (long long)Th * Tw), (long long)G * Th * Tw, G, -Hn, -Wn};
            if (!found || std::lexicographical_compare(key, key + 5, best, best + 5)) {
                std::copy(key, key + 5, best);
                found = true;
                I.Cn = Cn; I.G = G; I.Hn = Hn; I.Wn = Wn; I.th = th; I.tw = tw; I.Th = Th; I.Tw = Tw;
                I.Mn = Mn; I.Sout = (int)Sout;
            }
        }
    }
    if (!found) return false;
    I.T = I.Th * I.Tw;
    I.Ooff = (I.Cn - 1) * I.Hn * I.Wn + (s.h - 1) * I.Wn + s.h - 1;
    tiles.clear();
    for (int ti = 0; ti < I.Th; ti++)
        for (int tj = 0; tj < I.Tw; tj++) {
            const int a0 = ti * I.th, b0 = tj * I.tw;
            tiles.push_back({a0, std::min(Ho, a0 + I.th), b0, std::min(Wo, b0 + I.tw), a0, a0 + I.Hn, b0, b0 + I.Wn});
        }
    return true;
}

static void corr_tiles(const he_conv_shape &s, int th, int tw, std::vector<Tile> &tiles) {
    const int Ho = s.H + 2 * s.pad - s.h + 1, Wo = s.W + 2 * s.pad - s.h + 1;
    tiles.clear();
    for (int a0 = 0; a0 < Ho; a0 += th)
        for (int b0 = 0; b0 < Wo; b0 += tw) {
            const int a1 = std::min(Ho, a0 + th), b1 = std::min(Wo, b0 + tw);
            tiles.push_back({a0, a1, b0, b1, std::max(0, a0 - s.pad), std::min(s.H, a1 - s.pad + s.h - 1),
                             std::max(0, b0 - s.pad), std::min(s.W, b1 - s.pad + s.h - 1)});
        }
}

struct Geo { long long rlo, rhi, D1; };

static void corr_geometry(const he_conv_shape &s, const std::vector<Tile> &tiles, long long &O, long long &S,
                          std::vector<Geo> &g) {
    int Hm = 0, Wm = 0;
    for (const Tile &t : tiles) { Hm = std::max(Hm, t.r1 - t.r0); Wm = std::max(Wm, t.s1 - t.s0); }
    O = std::max(Hm, Wm) + s.h - 1;
    g.clear();
    S = 0;
    for (const Tile &t : tiles) {
        const long long ulo = t.a0 - s.pad - t.r0 + s.h - 1, uhi = t.a1 - 1 - s.pad - t.r0 + s.h - 1;
        const long long vlo = t.b0 - s.pad - t.s0 + s.h - 1, vhi = t.b1 - 1 - s.pad - t.s0 + s.h - 1;
        Geo e{ulo * O + vlo, uhi * O + vhi, (long long)(t.r1 - t.r0 + s.h - 2) * O + (t.s1 - t.s0 + s.h - 2)};
        S = std::max(S, std::max(e.rhi, e.D1 - e.rlo));
        g.push_back(e);
    }
    S += 1;
}

static bool corr_fits(long long c, long long S, const std::vector<Geo> &g, long long N) {
    for (const Geo &e : g) {
        if ((c - 1) * S + e.rhi >= N) return false;
        const long long D = 2 * (c - 1) * S + e.D1;
        if (!(D < N || D - N < (c - 1) * S + e.rlo)) return false;
    }
    return true;
}

static bool corr_search(int N, const he_conv_shape &s, bool dw, he_plan_info &I, std::vector<Tile> &tiles) {
    const int Ho = s.H + 2 * s.pad - s.h + 1, Wo = s.W + 2 * s.pad - s.h + 1;
    long long best[5] = {LLONG_MAX, 0, 0, 0, 0};
    bool found = false;
    std::vector<Tile> tl;
    std::vector<Geo> g;
    for (int th = 1; th <= Ho; th++)
        for (int tw = 1; tw <= Wo; tw++) {
            corr_tiles(s, th, tw, tl);
            long long O, S;
            corr_geometry(s, tl, O, S, g);
            if (!corr_fits(1, S, g, N)) continue;
            int cmax = 1;
            while (cmax < s.C && corr_fits(cmax + 1, S, g, N)) cmax++;
            // every channel count up to the largest that fits: fewer channels
            // per polynomial can leave room for more kernels per polynomial
            int last_G = -1;
            for (int ct = cmax; ct >= 1; ct--) {
                const int G = (s.C + ct - 1) / ct;
                if (G == last_G) continue;
                last_G = G;
                const int Cn = (s.C + G - 1) / G;
                std::vector<Span> sp;
                for (const Geo &e : g)
                    sp.push_back({(Cn - 1) * S + e.rlo, (Cn - 1) * S + e.rhi, 2 * (long long)(Cn - 1) * S + e.D1});
                int Mn;
                long long Sout;
                out_packing(s.M, N, sp, Mn, Sout, dw && G > 1 ? Cn : 0);
                const long long MG = (s.M + Mn - 1) / Mn;
                long long key[5] = {plan_products(dw, MG, G, (long long)tl.size()), (long long)G * (long long)tl.size(),
                                    G, -th, -tw};
                if (!found || std::lexicographical_compare(key, key + 5, best, best + 5)) {
                    std::copy(key, key + 5, best);
                    found = true;
                    I.Cn = Cn; I.G = G; I.th = th; I.tw = tw; I.O = (int)O; I.S = (int)S;
                    I.Th = (Ho + th - 1) / th; I.Tw = (Wo + tw - 1) / tw;
                    I.Mn = Mn; I.Sout = (int)Sout;
                    tiles = tl;
                }
            }
        }
    if (!found) return false;
    I.T = I.Th * I.Tw;
    return true;
}

// The window and output-packing search alone (no maps).
static int search_plan(int N, const he_conv_shape &s, int encoding, he_plan_info &I, std::vector<Tile> &tiles,
                       std::string &err) {
    if (s.C < 1 || s.H < 1 || s.W < 1 || s.M < 1 || s.h < 1 || s.pad < 0 || s.pad > s.h - 1 ||
        s.H + 2 * s.pad - s.h + 1 < 1 || s.W + 2 * s.pad - s.h + 1 < 1) {
        err = "bad convolution shape";
        return HE_ERR_INVALID_ARG;
    }
    const bool dw = (encoding & HE_PLAN_DEPTHWISE) != 0;
    encoding &= ~HE_PLAN_DEPTHWISE;
    if (encoding != HE_ENC_CONVENTIONAL && encoding != HE_ENC_CORRELATED) { err = "bad encoding"; return HE_ERR_INVALID_ARG; }
    if (dw && s.M != s.C) { err = "a depthwise layer has as many output channels as input channels"; return HE_ERR_INVALID_ARG; }
    if (N < 2 || (N & (N - 1))) { err = "N must be a power of two"; return HE_ERR_INVALID_ARG; }
    memset(&I, 0, sizeof I);
    I.encoding = encoding;
    I.depthwise = dw ? 1 : 0;
    I.Ho = s.H + 2 * s.pad - s.h + 1;
    I.Wo = s.W + 2 * s.pad - s.h + 1;
    const bool ok = encoding == HE_ENC_CONVENTIONAL ? conv_search(N, s, dw, I, tiles) : corr_search(N, s, dw, I, tiles);
    if (!ok) { err = "no partition window fits the ring"; return HE_ERR_PLAN_DOES_NOT_FIT; }
    I.MG = (s.M + I.Mn - 1) / I.Mn;
    return HE_OK;
}

int build_plan(he_ctx *c, const he_conv_shape &s, int encoding, he_plan *p, std::string &err) {
    const int N = c->N;
    he_plan_info I;
    std::vector<Tile> tiles;
    const int rc = search_plan(N, s, encoding, I, tiles, err);
    if (rc) return rc;
    encoding = I.encoding;  // without the depthwise flag
    p->s = s;
    p->info = I;
    p->N = N;
    p->tiles.clear();
    for (const Tile &t : tiles) {
        int v[8] = {t.a0, t.a1, t.b0, t.b1, t.r0, t.r1, t.s0, t.s1};
        p->tiles.insert(p->tiles.end(), v, v + 8);
    }
    // index maps
    I.MG = (s.M + I.Mn - 1) / I.Mn;
    p->info = I;
    const int T = I.T, G = I.G, Cn = I.Cn, MG = I.MG, HW = I.Ho * I.Wo;
    p->h_in_map.assign((size_t)T * G * N, -1);
    p->h_ker_map.assign((size_t)MG * G * N, -1);
    p->h_out_map.assign((size_t)s.M * HW, -1);
    for (int ti = 0; ti < T; ti++) {
        const Tile &t = tiles[ti];
        for (int g = 0; g < G; g++) {
            int32_t *m = p->h_in_map.data() + ((size_t)ti * G + g) * N;
            for (int cl = 0; cl < Cn; cl++) {
                const int ch = g * Cn + cl;
                if (ch >= s.C) break;
                if (encoding == HE_ENC_CONVENTIONAL) {
                    for (int i = 0; i < I.Hn; i++)
                        for (int j = 0; j < I.Wn; j++) {
                            const int r = t.r0 + i - s.pad, q = t.s0 + j - s.pad;
                            if (r >= 0 && r < s.H && q >= 0 && q < s.W)
                                m[cl * I.Hn * I.Wn + i * I.Wn + j] = (ch * s.H + r) * s.W + q;
                        }
                } else {
                    for (int i = t.r0; i < t.r1; i++)
                        for (int j = t.s0; j < t.s1; j++)
                            m[(long long)cl * I.S + (long long)(i - t.r0) * I.O + (j - t.s0)] = (ch * s.H + i) * s.W + j;
                }
            }
        }
        for (int a = t.a0; a < t.a1; a++)
            for (int b = t.b0; b < t.b1; b++) {
                long long coef;
                if (encoding == HE_ENC_CONVENTIONAL) coef = I.Ooff + (long long)(a - t.a0) * I.Wn + (b - t.b0);
                else {
                    const long long u = a - s.pad - t.r0 + s.h - 1, v = b - s.pad - t.s0 + s.h - 1;
                    coef = (long long)(Cn - 1) * I.S + u * I.O + v;
                }
                for (int mo = 0; mo < s.M; mo++)
                    p->h_out_map[(size_t)mo * HW + (size_t)a * I.Wo + b] =
                        (int32_t)(((long long)(mo / I.Mn) * T + ti) * N + coef + (long long)(mo % I.Mn) * I.Sout);
            }
    }
    for (int mo = 0; mo < s.M; mo++)
        for (int g = 0; g < G; g++) {
            int32_t *m = p->h_ker_map.data() + ((size_t)(mo / I.Mn) * G + g) * N;
            const long long off = (long long)(mo % I.Mn) * I.Sout;
            for (int cl = 0; cl < Cn; cl++) {
                const int ch = g * Cn + cl;
                if (ch >= s.C) break;
                for (int k = 0; k < s.h; k++)
                    for (int l = 0; l < s.h; l++) {
                        long long coef = encoding == HE_ENC_CONVENTIONAL
                            ? (long long)I.Ooff - (long long)cl * I.Hn * I.Wn - (long long)k * I.Wn - l
                            : (long long)(Cn - 1 - cl) * I.S + (long long)(s.h - 1 - k) * I.O + (s.h - 1 - l);
                        m[coef + off] = ((mo * s.C + ch) * s.h + k) * s.h + l;
                    }
            }
        }
    // upload
    auto up = [&](const std::vector<int32_t> &h, int32_t **d) -> bool {
        if (he::dev_alloc((void **)d, h.size() * 4) != cudaSuccess) return false;
        return cudaMemcpy(*d, h.data(), h.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (!up(p->h_in_map, &p->in_map) || !up(p->h_ker_map, &p->ker_map) || !up(p->h_out_map, &p->out_map)) {
        err = "upload plan maps";
        return HE_ERR_OOM;
    }
    return HE_OK;
}

}  // namespace he

extern "C" int he_plan_search(int N, const he_conv_shape *shape, int encoding, he_plan_info *info) {
    if (!shape || !info) return HE_ERR_INVALID_ARG;
    he_plan_info I;
    std::vector<he::Tile> tiles;
    std::string err;
    const int rc = he::search_plan(N, *shape, encoding, I, tiles, err);
    if (!rc) *info = I;
    return rc;
}
