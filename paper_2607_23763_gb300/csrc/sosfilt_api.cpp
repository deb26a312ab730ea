// C ABI of libsosfilt.so (declared in include/sosfilt.h): filter objects,
// the float64 host precompute of the per-section tables (Sec. II-C..F), the
// library-owned lookback workspace, and the launch of one kernel pass per
// group of up to eight sections.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "sosfilt.h"
#include "sosfilt_internal.h"

namespace sosk {
bool dccr_available(int K, int N, bool norm, int lbm);
int cascade_blocks_per_sm_32(int K, bool norm);
int cascade_blocks_per_sm_64(int K, bool norm);
size_t cascade_smem_32(int K);
size_t cascade_smem_64(int K);
int cascade_blocks_per_sm(int K, int N, bool norm) {
    return N == 32 ? cascade_blocks_per_sm_32(K, norm) : N == 64 ? cascade_blocks_per_sm_64(K, norm) : 0;
}
int cascade_warps(int N) { return N == 32 ? 8 : 4; }
size_t cascade_smem(int K, int N) { return N == 32 ? cascade_smem_32(K) : N == 64 ? cascade_smem_64(K) : 0; }
int lane_blocks_per_sm_n32a(int K, bool norm);
int lane_blocks_per_sm_n32b(int K, bool norm);
int lane_blocks_per_sm_n64a(int K, bool norm);
int lane_blocks_per_sm_n64b(int K, bool norm);
int lane_blocks_per_sm_n64w10a(int K, bool norm);
int lane_blocks_per_sm_n64w10b(int K, bool norm);
int lane_blocks_per_sm(int K, int N, int W, bool norm) {
    if (N == 32) return K <= 4 ? lane_blocks_per_sm_n32a(K, norm) : lane_blocks_per_sm_n32b(K, norm);
    if (W == kLaneWide) return K <= 4 ? lane_blocks_per_sm_n64w10a(K, norm) : lane_blocks_per_sm_n64w10b(K, norm);
    return K <= 4 ? lane_blocks_per_sm_n64a(K, norm) : lane_blocks_per_sm_n64b(K, norm);
}
}  // namespace sosk

namespace {

constexpr int kNumN = 3;
constexpr int kSupportedN[kNumN] = {32, 64, 128};
constexpr long long kDefaultSpinBudget = 2000000000LL;  // ~1 s of SM clock

struct Mat {
    double a, b, c, d;  // row-major 2x2
};

Mat mul(const Mat &x, const Mat &y) {
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}

Mat mpow(Mat m, long long e) {
    Mat r{1, 0, 0, 1};
    while (e > 0) {
        if (e & 1) r = mul(r, m);
        m = mul(m, m);
        e >>= 1;
    }
    return r;
}

std::vector<double> polymul(const std::vector<double> &p, const std::vector<double> &q) {
    std::vector<double> r(p.size() + q.size() - 1, 0.0);
    for (size_t i = 0; i < p.size(); ++i)
        for (size_t j = 0; j < q.size(); ++j) r[i + j] += p[i] * q[j];
    return r;
}

int ilog2i(int n) {
    int d = 0;
    while ((1 << d) < n) ++d;
    return d;
}

struct NTables {
    int N = 0;
    std::vector<sosk::SecCoef> sec;  // [K]
    float4 *d_lane_pow = nullptr;    // [K][32]
    float4 *d_grp_pow = nullptr;     // [K][kGrpPowStride]: powers of T^C
    float4 *d_cta_pow = nullptr;     // [K][kGrpPowStride]: powers of the block transition T^(kWarps C)
};

// Dense float64 matrices acting on the cascade state (2K words, section-major, (z1, z2) each).
struct DMat {
    int n = 0;
    std::vector<double> a;
    explicit DMat(int n_ = 0) : n(n_), a(static_cast<size_t>(n_) * n_, 0.0) {}
    double &at(int i, int j) { return a[static_cast<size_t>(i) * n + j]; }
    double at(int i, int j) const { return a[static_cast<size_t>(i) * n + j]; }
};

DMat deye(int n) {
    DMat r(n);
    for (int i = 0; i < n; ++i) r.at(i, i) = 1.0;
    return r;
}

DMat dmul(const DMat &x, const DMat &y) {
    DMat r(x.n);
    for (int i = 0; i < x.n; ++i)
        for (int k = 0; k < x.n; ++k) {
            const double v = x.at(i, k);
            if (v == 0.0) continue;
            for (int j = 0; j < x.n; ++j) r.at(i, j) += v * y.at(k, j);
        }
    return r;
}

DMat dpow(DMat m, long long e) {
    DMat r = deye(m.n);
    while (e > 0) {
        if (e & 1) r = dmul(r, m);
        m = dmul(m, m);
        e >>= 1;
    }
    return r;
}

// One pass (<= 8 sections) of the cascade-carry kernel for one N.
struct CasPass {
    int k0 = 0, kp = 0;
    std::vector<double> coef;  // [kp][5] b0, b1, b2, a1, a2 as the kernel applies them
    DMat M1;                   // one-sample zero-input transition of the pass's cascade state
    std::vector<float> H;      // [2 kp][N] zero-input output basis
    float *d_tab = nullptr;    // device table block (CasDims<kp>::TAB floats)
    long long tail_p = -1;     // position for which A_tail is cached
    std::vector<float> A_tail; // packed transition over tail_p + 1 samples
};

struct CasTables {
    int N = 0;
    std::vector<CasPass> passes;
};

// One pass (<= 8 sections) of the skewed-pass PH kernel (sosfilt_lane.cuh) for one N.
struct LanePass {
    int k0 = 0, kp = 0, N = 0, W = 0;  // sections k0 .. k0 + kp - 1; N samples per lane, W groups per tile
    std::vector<double> coef;        // [kp][5] as the kernel applies them
    DMat M1;                         // one-sample zero-input transition of the pass's cascade state
    std::vector<sosk::LaneSec> sec;  // [kp]
    std::vector<float> MX;           // coupling blocks of M_N, row-major 2x2, kp (kp - 1) / 2 of them
    std::vector<float> H;            // [2 kp][N] zero-input output basis
    float *d_tab = nullptr;          // device table block (LaneDims<kp, N>::TAB_GLOBAL floats)
    // the cascade transition over the first m + 1 samples of a lane, M1^(m+1) packed, m < N: the
    // final state's tail transition, taken by every run without further host work
    std::vector<float> Mm;           // [N][packed_floats(kp)]
    // the batch kernel's geometries (N = kBatchN or kBatchNs, W = kBatchW) only: device copies for
    // the multi-signal kernel
    sosk::LaneSec *d_sec = nullptr;  // [kp] section constants
    float4 *d_MX = nullptr;          // coupling blocks of M_N
    float *d_Mm = nullptr;           // device copy of Mm
    // tensor-core kernel only (N = 64, W = kTcGroups): its constant operands and final-state table
    float *d_tcimg = nullptr;        // shared-memory image of the MMA B operands (kTcImageBytes)
    float *d_gtail = nullptr;        // [2 kp][64] state responses G, float32
};

}  // namespace

// What a batched run reads of a filter, in one cache line at the front of the filter object: the
// batch kernel's device tables for each tile geometry (first pass; the transition powers M1^(m+1),
// m < 64, serve both) and the launch class.
struct BatchTmpl {
    const sosk::LaneSec *sec[sosk::kBatchGeoms] = {};
    const float4 *MX[sosk::kBatchGeoms] = {};
    const float *tab[sosk::kBatchGeoms] = {};
    const float *Mm = nullptr;
    float gain = 1.f;
    short cls = -1;        // (K - 1) * 2 + b0-normalized (geometry 0), or -1 for more than kMaxPass sections
    signed char geom = -1;  // tile geometry pinned by the filter's tuning (N = 64: 0, N = 32: 1), or -1
};
static_assert(sizeof(BatchTmpl) <= 64, "one cache line");

struct sos_filter {
    int K = 0;
    int device = 0;
    BatchTmpl bt;
    std::vector<double> sos;  // [K][5]
    bool norm = false;
    double gain = 1.0;
    std::vector<double> zscale;  // [K]
    sos_tuning tuning{};
    NTables tables[kNumN];
    CasTables cas[2];  // N = 32, 64
    // PH kernels: skewed pass at (N, W) = (32, 7), (64, 7), (64, 10); tensor cores at (64, 8)
    std::vector<LanePass> lane[4];
    // workspace
    unsigned long long *d_desc = nullptr;
    size_t desc_groups = 0;  // capacity in groups (per section slot)
    unsigned long long *d_ticket = nullptr;  // [2]: eager launches' counter, captured launches' counter
    unsigned long long ticket_base = 0;
    unsigned int epoch = 0;
    int *d_status = nullptr;
    float *d_state = nullptr;  // resident [K][2]
    cudaStream_t last_stream = nullptr;
    unsigned long long *trace = nullptr;
    long long trace_blocks = 0;
    // host-buffer pipeline (sos_filter_run_host), created on first use
    cudaStream_t hs[3] = {nullptr, nullptr, nullptr};  // copy in, filter, copy out
    cudaEvent_t ev_in[3] = {}, ev_done[3] = {}, ev_out[3] = {};
    float *hbuf[3] = {nullptr, nullptr, nullptr};
    long long hbuf_samples = 0;
    float *d_hstate = nullptr;  // [K][2]
    std::mutex mu;
};

namespace {

sos_status cuda_fail() { return SOS_ECUDA; }

bool section_stable(double a1, double a2) { return std::fabs(a2) < 1.0 && std::fabs(a1) < 1.0 + a2; }

// Per-section tables for one N, float64 -> float32 once.
void build_tables(sos_filter *f, int N, NTables &t, std::vector<float4> &lane_pow, std::vector<float4> &grp_pow,
                  std::vector<float4> &cta_pow) {
    const int D = ilog2i(N);
    t.N = N;
    t.sec.assign(f->K, sosk::SecCoef{});
    lane_pow.assign(static_cast<size_t>(f->K) * 32, float4{});
    grp_pow.assign(static_cast<size_t>(f->K) * sosk::kGrpPowStride, float4{});
    cta_pow.assign(static_cast<size_t>(f->K) * sosk::kGrpPowStride, float4{});
    for (int k = 0; k < f->K; ++k) {
        const double *c = &f->sos[5 * k];
        double b0 = c[0], b1 = c[1], b2 = c[2];
        const double a1 = c[3], a2 = c[4];
        if (f->norm) {
            b1 /= b0;
            b2 /= b0;
            b0 = 1.0;
        }
        sosk::SecCoef &s = t.sec[k];
        std::memset(&s, 0, sizeof s);
        const std::vector<double> taps = polymul({b0, b1, b2}, {1.0, -a1, a2});  // B(z) A(-z)
        s.t0 = static_cast<float>(taps[0]);
        s.t1 = static_cast<float>(taps[1]);
        s.t2 = static_cast<float>(taps[2]);
        s.t3 = static_cast<float>(taps[3]);
        s.t4 = static_cast<float>(taps[4]);
        s.b1 = static_cast<float>(b1);
        s.b2 = static_cast<float>(b2);
        s.a1 = static_cast<float>(a1);
        s.a2 = static_cast<float>(a2);
        // level coefficients: e_0 = a1, f_0 = a2, e_{i+1} = 2 f_i - e_i^2, f_{i+1} = f_i^2
        std::vector<double> e(D + 1), fl(D + 1);
        e[0] = a1;
        fl[0] = a2;
        for (int i = 0; i < D; ++i) {
            e[i + 1] = 2.0 * fl[i] - e[i] * e[i];
            fl[i + 1] = fl[i] * fl[i];
        }
        for (int i = 1; i < D; ++i) {
            s.ne[i] = static_cast<float>(-e[i]);
            s.f[i] = static_cast<float>(fl[i]);
            s.nf[i] = static_cast<float>(-fl[i]);
        }
        // state injection: Q_i = prod_{j<i} (1 - e_j z^-(2^j) + f_j z^-(2^(j+1)))
        std::vector<double> Q{1.0};
        for (int i = 0; i < D; ++i) {
            const int st = 1 << i;
            std::vector<double> g(2 * st + 1, 0.0);
            g[0] = 1.0;
            g[st] = -e[i];
            g[2 * st] = fl[i];
            Q = polymul(Q, g);
            const int lev = i + 1;
            auto q = [&](int m) { return (m >= 0 && m < static_cast<int>(Q.size())) ? Q[m] : 0.0; };
            const int mo = (1 << lev) - 1, me = (1 << lev) - 2;
            s.qo[lev][0] = static_cast<float>(q(mo));
            s.qo[lev][1] = static_cast<float>(q(mo - 1));
            s.qe[lev][0] = static_cast<float>(q(me));
            s.qe[lev][1] = static_cast<float>(q(me - 1));
        }
        // transitions of the transposed direct form II state over N and C = 32 N samples
        const Mat T{-a1, 1.0, -a2, 0.0};
        const Mat TN = mpow(T, N);
        Mat P = TN;
        for (int kk = 0; kk < 5; ++kk) {
            s.tn[kk][0] = static_cast<float>(P.a);
            s.tn[kk][1] = static_cast<float>(P.b);
            s.tn[kk][2] = static_cast<float>(P.c);
            s.tn[kk][3] = static_cast<float>(P.d);
            P = mul(P, P);
        }
        Mat L{1, 0, 0, 1};
        for (int l = 0; l < 32; ++l) {
            lane_pow[static_cast<size_t>(k) * 32 + l] =
                float4{static_cast<float>(L.a), static_cast<float>(L.b), static_cast<float>(L.c), static_cast<float>(L.d)};
            L = mul(L, TN);
        }
        const Mat TC = L;  // TN^32
        {
            Mat W{1, 0, 0, 1};
            for (int w = 0; w <= sosk::kWarps; ++w) {
                s.tc[w][0] = static_cast<float>(W.a);
                s.tc[w][1] = static_cast<float>(W.b);
                s.tc[w][2] = static_cast<float>(W.c);
                s.tc[w][3] = static_cast<float>(W.d);
                W = mul(W, TC);
            }
        }
        // powers S^k (k = 0..32) and S^(32 i) (i = 0..16) of a step matrix S
        auto fill = [&](std::vector<float4> &tab, const Mat &S) {
            auto put = [&](int idx, const Mat &m) {
                tab[static_cast<size_t>(k) * sosk::kGrpPowStride + idx] = float4{
                    static_cast<float>(m.a), static_cast<float>(m.b), static_cast<float>(m.c), static_cast<float>(m.d)};
            };
            Mat Gp{1, 0, 0, 1};
            for (int j = 0; j <= 32; ++j) {
                put(j, Gp);
                Gp = mul(Gp, S);
            }
            const Mat S32 = mpow(S, 32);
            Mat G32{1, 0, 0, 1};
            for (int i = 0; i <= sosk::kMaxLBM; ++i) {
                put(sosk::kPow32 + i, G32);
                G32 = mul(G32, S32);
            }
        };
        fill(grp_pow, TC);
        fill(cta_pow, mpow(TC, sosk::kWarps));
        s.zscale = static_cast<float>(f->zscale[k]);
        s.zscale_inv = static_cast<float>(1.0 / f->zscale[k]);
        auto dup = [](float v) { return float2{v, v}; };
        s.p_t0 = dup(s.t0);
        s.p_t1 = dup(s.t1);
        s.p_t2 = dup(s.t2);
        s.p_t3 = dup(s.t3);
        s.p_t4 = dup(s.t4);
        for (int i = 0; i <= sosk::kMaxD; ++i) {
            s.p_ne[i] = dup(s.ne[i]);
            s.p_f[i] = dup(s.f[i]);
            s.p_nf[i] = dup(s.nf[i]);
            s.p_q0[i] = float2{s.qe[i][0], s.qo[i][0]};
            s.p_q1[i] = float2{s.qe[i][1], s.qo[i][1]};
        }
    }
}

// Zero-input step of a cascade with coefficients c[kp][5] (as applied in the kernel's domain).
double cascade_step(const std::vector<double> &c, int kp, std::vector<double> &z, double x) {
    double v = x;
    for (int s = 0; s < kp; ++s) {
        const double *q = &c[5 * s];
        const double y = q[0] * v + z[2 * s];
        const double z1 = q[1] * v - q[3] * y + z[2 * s + 1];
        const double z2 = q[2] * v - q[4] * y;
        z[2 * s] = z1;
        z[2 * s + 1] = z2;
        v = y;
    }
    return v;
}

// Packed lower block-triangular storage: block (s, t), s >= t, at 4 (s(s+1)/2 + t), row-major 2x2.
void pack_into(const DMat &m, int kp, float *dst) {
    for (int s = 0; s < kp; ++s)
        for (int t = 0; t <= s; ++t) {
            float *b = dst + 4 * (s * (s + 1) / 2 + t);
            b[0] = static_cast<float>(m.at(2 * s, 2 * t));
            b[1] = static_cast<float>(m.at(2 * s, 2 * t + 1));
            b[2] = static_cast<float>(m.at(2 * s + 1, 2 * t));
            b[3] = static_cast<float>(m.at(2 * s + 1, 2 * t + 1));
        }
}

int packed_floats(int kp) { return 2 * kp * (kp + 1); }
int lane_stride(int kp) {
    const int nf = packed_floats(kp);
    return ((nf / 4) & 1) ? nf : nf + 4;
}
// Table block of one pass: (M_N)^lane [32][stride], (A_T)^lane [32][stride] (packed), A_C dense
// column-major (these are copied to shared memory), then A_T dense and (A_T)^(32 w) dense for
// w = 1..kMaxWin (read from global memory).
int table_floats(int kp) {
    const int full = (2 * kp) * (2 * kp);
    return 2 * 32 * lane_stride(kp) + 2 * full + sosk::kMaxWin * full;
}

void dense_colmajor_into(const DMat &m, float *dst) {
    for (int j = 0; j < m.n; ++j)
        for (int i = 0; i < m.n; ++i) dst[static_cast<size_t>(j) * m.n + i] = static_cast<float>(m.at(i, j));
}

int table_index(int N);

// Transitions and output basis of every pass for one N, in float64, uploaded once.
sos_status build_cascade(sos_filter *f, int N, CasTables &ct) {
    ct.N = N;
    ct.passes.clear();
    const int W = sosk::cascade_warps(N);
    for (int k0 = 0; k0 < f->K; k0 += sosk::kMaxPass) {
        CasPass ps;
        ps.k0 = k0;
        ps.kp = (f->K - k0) < sosk::kMaxPass ? (f->K - k0) : sosk::kMaxPass;
        const int kp = ps.kp, S = 2 * kp;
        ps.coef.resize(5 * kp);
        for (int j = 0; j < kp; ++j) {
            const double *c = &f->sos[5 * (k0 + j)];
            double b0 = c[0], b1 = c[1], b2 = c[2];
            if (f->norm) {
                b1 /= b0;
                b2 /= b0;
                b0 = 1.0;
            }
            ps.coef[5 * j + 0] = b0;
            ps.coef[5 * j + 1] = b1;
            ps.coef[5 * j + 2] = b2;
            ps.coef[5 * j + 3] = c[3];
            ps.coef[5 * j + 4] = c[4];
        }
        ps.M1 = DMat(S);
        ps.H.assign(static_cast<size_t>(S) * N, 0.f);
        for (int j = 0; j < S; ++j) {
            std::vector<double> z(S, 0.0);
            z[j] = 1.0;
            cascade_step(ps.coef, kp, z, 0.0);
            for (int i = 0; i < S; ++i) ps.M1.at(i, j) = z[i];
            std::vector<double> h(S, 0.0);
            h[j] = 1.0;
            for (int m = 0; m < N; ++m) ps.H[static_cast<size_t>(j) * N + m] = static_cast<float>(cascade_step(ps.coef, kp, h, 0.0));
        }
        const DMat MN = dpow(ps.M1, N);
        const DMat AC = dpow(MN, 32);
        const DMat AT = dpow(AC, W);
        const int ms = lane_stride(kp), full = S * S;
        std::vector<float> tab(table_floats(kp), 0.f);
        DMat L = deye(S), LT = deye(S);
        for (int l = 0; l < 32; ++l) {
            pack_into(L, kp, &tab[static_cast<size_t>(l) * ms]);
            pack_into(LT, kp, &tab[static_cast<size_t>(32 + l) * ms]);
            L = dmul(L, MN);
            LT = dmul(LT, AT);
        }
        float *p_dense = &tab[64 * static_cast<size_t>(ms)];
        dense_colmajor_into(AC, p_dense);
        dense_colmajor_into(AT, p_dense + full);
        const DMat AT32 = dpow(AT, 32);
        DMat Pw = AT32;
        for (int w = 1; w <= sosk::kMaxWin; ++w) {
            dense_colmajor_into(Pw, p_dense + full * (1 + w));
            Pw = dmul(Pw, AT32);
        }
        if (cudaMalloc(&ps.d_tab, tab.size() * sizeof(float)) != cudaSuccess) return SOS_ENOMEM;
        if (cudaMemcpy(ps.d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return SOS_ECUDA;
        ct.passes.push_back(std::move(ps));
    }
    return SOS_OK;
}

// Tables of the skewed-pass PH kernel for one N (32 or 64), in float64, uploaded once.  Layout of
// the device block as LaneDims<kp, N>: (M_N)^lane [32][stride], (A_T)^lane [32][stride] (packed),
// A_C dense column-major, the output basis [2 kp][N], A_T dense.
sos_status build_lane(sos_filter *f, int N, int W, std::vector<LanePass> &out) {
    out.clear();
    for (int k0 = 0; k0 < f->K; k0 += sosk::kMaxPass) {
        LanePass ps;
        ps.k0 = k0;
        ps.N = N;
        ps.W = W;
        ps.kp = (f->K - k0) < sosk::kMaxPass ? (f->K - k0) : sosk::kMaxPass;
        const int kp = ps.kp, S = 2 * kp;
        ps.coef.resize(5 * kp);
        for (int j = 0; j < kp; ++j) {
            const double *c = &f->sos[5 * (k0 + j)];
            double b0 = c[0], b1 = c[1], b2 = c[2];
            if (f->norm) {
                b1 /= b0;
                b2 /= b0;
                b0 = 1.0;
            }
            ps.coef[5 * j + 0] = b0;
            ps.coef[5 * j + 1] = b1;
            ps.coef[5 * j + 2] = b2;
            ps.coef[5 * j + 3] = c[3];
            ps.coef[5 * j + 4] = c[4];
        }
        ps.M1 = DMat(S);
        ps.H.assign(static_cast<size_t>(S) * N, 0.f);
        for (int j = 0; j < S; ++j) {
            std::vector<double> z(S, 0.0);
            z[j] = 1.0;
            cascade_step(ps.coef, kp, z, 0.0);
            for (int i = 0; i < S; ++i) ps.M1.at(i, j) = z[i];
            std::vector<double> h(S, 0.0);
            h[j] = 1.0;
            for (int m = 0; m < N; ++m)
                ps.H[static_cast<size_t>(j) * N + m] = static_cast<float>(cascade_step(ps.coef, kp, h, 0.0));
        }
        const DMat MN = dpow(ps.M1, N);
        const DMat AC = dpow(MN, 32);
        const DMat AT = dpow(AC, W);
        auto f32 = [](double v) { return static_cast<float>(v); };
        ps.sec.assign(kp, sosk::LaneSec{});
        for (int j = 0; j < kp; ++j) {
            sosk::LaneSec &c = ps.sec[j];
            const double b0 = ps.coef[5 * j], b1 = ps.coef[5 * j + 1], b2 = ps.coef[5 * j + 2];
            const double a1 = ps.coef[5 * j + 3], a2 = ps.coef[5 * j + 4];
            c.c = float4{f32(b1), f32(b2), f32(-a1), f32(-a2)};
            Mat P{MN.at(2 * j, 2 * j), MN.at(2 * j, 2 * j + 1), MN.at(2 * j + 1, 2 * j), MN.at(2 * j + 1, 2 * j + 1)};
            for (int r = 0; r < 5; ++r) {
                c.tn[r] = float4{f32(P.a), f32(P.b), f32(P.c), f32(P.d)};
                P = mul(P, P);
            }
            c.b0 = f32(b0);
            c.zscale = f32(f->zscale[k0 + j]);
            c.zscale_inv = f32(1.0 / f->zscale[k0 + j]);
        }
        ps.MX.assign(kp > 1 ? 2 * kp * (kp - 1) : 4, 0.f);
        for (int k = 1; k < kp; ++k)
            for (int j = 0; j < k; ++j) {
                float *b = &ps.MX[4 * (k * (k - 1) / 2 + j)];
                b[0] = f32(MN.at(2 * k, 2 * j));
                b[1] = f32(MN.at(2 * k, 2 * j + 1));
                b[2] = f32(MN.at(2 * k + 1, 2 * j));
                b[3] = f32(MN.at(2 * k + 1, 2 * j + 1));
            }
        const int ms = lane_stride(kp), full = S * S;
        const size_t off_ac = 64 * static_cast<size_t>(ms), off_h = off_ac + full, off_at = off_h + N * S;
        const size_t off_at32 = off_at + full, off_at31 = off_at32 + full, off_acp = off_at31 + full;
        std::vector<float> tab(off_acp + static_cast<size_t>(W - 1) * full, 0.f);
        DMat L = deye(S), LT = deye(S);
        for (int l = 0; l < 32; ++l) {
            pack_into(L, kp, &tab[static_cast<size_t>(l) * ms]);
            pack_into(LT, kp, &tab[static_cast<size_t>(32 + l) * ms]);
            L = dmul(L, MN);
            LT = dmul(LT, AT);
        }
        dense_colmajor_into(AC, &tab[off_ac]);
        for (int j = 0; j < S; ++j)
            for (int m = 0; m < N; ++m) tab[off_h + static_cast<size_t>(j) * N + m] = ps.H[static_cast<size_t>(j) * N + m];
        dense_colmajor_into(AT, &tab[off_at]);
        dense_colmajor_into(dpow(AT, 32), &tab[off_at32]);
        dense_colmajor_into(dpow(AT, 31), &tab[off_at31]);
        {
            DMat P = AC;
            for (int v = 1; v < W; ++v) {
                dense_colmajor_into(P, &tab[off_acp + static_cast<size_t>(v - 1) * full]);
                P = dmul(P, AC);
            }
        }
        if (cudaMalloc(&ps.d_tab, tab.size() * sizeof(float)) != cudaSuccess) return SOS_ENOMEM;
        if (cudaMemcpy(ps.d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return SOS_ECUDA;
        const int nf = packed_floats(kp);
        ps.Mm.assign(static_cast<size_t>(N) * nf, 0.f);
        DMat Pm = ps.M1;
        for (int m = 0; m < N; ++m) {
            pack_into(Pm, kp, &ps.Mm[static_cast<size_t>(m) * nf]);
            Pm = dmul(Pm, ps.M1);
        }
        if ((N == sosk::kBatchN || N == sosk::kBatchNs) && W == sosk::kBatchW) {
            const std::vector<float> &mm = ps.Mm;
            const bool with_mm = N == sosk::kBatchN;  // M1^(m+1) for m < 64 serves both geometries
            if (cudaMalloc(&ps.d_sec, sizeof(sosk::LaneSec) * kp) != cudaSuccess ||
                cudaMalloc(&ps.d_MX, sizeof(float) * ps.MX.size()) != cudaSuccess ||
                (with_mm && cudaMalloc(&ps.d_Mm, sizeof(float) * mm.size()) != cudaSuccess))
                return SOS_ENOMEM;
            if (cudaMemcpy(ps.d_sec, ps.sec.data(), sizeof(sosk::LaneSec) * kp, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(ps.d_MX, ps.MX.data(), sizeof(float) * ps.MX.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                (with_mm && cudaMemcpy(ps.d_Mm, mm.data(), sizeof(float) * mm.size(), cudaMemcpyHostToDevice) != cudaSuccess))
                return SOS_ECUDA;
        }
        out.push_back(std::move(ps));
    }
    return SOS_OK;
}

// Operands of the tensor-core kernel for one pass (Sec. II-C with the particular solution as a
// product): the pass's cascade, as the tables model it (b0-normalized sections, the input gain in the
// first pass), driven by an impulse gives the impulse response h and the state responses; the
// particular solution of a 64-sample row is T x with T[m][j] = h[m - j] (m >= j), the row's terminal
// state G x with G[s][j] the state s after sample 63 of an impulse at j.  B1 stacks T (rows 0..63)
// and G (rows 64..64 + 2 kp - 1) as 80 rows over the 64 input samples; B2 holds the zero-input output
// basis H[m][s].  Each value is split into its TF32 head (upper 19 bits of the float32) and the
// float32 remainder, laid out as the kernel's shared memory holds them: K-major rows of 128 bytes
// whose 16-byte chunk j sits at chunk j ^ (row mod 8).
sos_status build_tc(sos_filter *f, LanePass &ps) {
    constexpr int N = 64, R1 = 80, HB = 2 * R1 * 128;  // samples per row, B1 rows, bytes of one B1 image
    const int kp = ps.kp, S = 2 * kp;
    const double gain = ps.k0 == 0 ? f->gain : 1.0;
    std::vector<double> h(N), g(static_cast<size_t>(N) * S);
    {
        std::vector<double> z(S, 0.0);
        for (int m = 0; m < N; ++m) {
            h[m] = cascade_step(ps.coef, kp, z, m == 0 ? gain : 0.0);
            for (int k = 0; k < S; ++k) g[static_cast<size_t>(m) * S + k] = z[k];
        }
    }
    std::vector<double> H(static_cast<size_t>(S) * N);
    for (int k = 0; k < S; ++k) {
        std::vector<double> z(S, 0.0);
        z[k] = 1.0;
        for (int m = 0; m < N; ++m) H[static_cast<size_t>(k) * N + m] = cascade_step(ps.coef, kp, z, 0.0);
    }
    std::vector<unsigned char> img(sosk::kTcImageBytes, 0);
    auto put = [&](size_t base, int r, int c, float v) {
        const size_t off = base + static_cast<size_t>(r) * 128 + ((((c >> 2) ^ (r & 7)) << 4) | ((c & 3) << 2));
        std::memcpy(&img[off], &v, sizeof v);
    };
    auto head = [](double v) {
        float x = static_cast<float>(v);
        uint32_t u;
        std::memcpy(&u, &x, sizeof u);
        u &= 0xffffe000u;
        std::memcpy(&x, &u, sizeof x);
        return x;
    };
    for (int n = 0; n < R1; ++n)
        for (int j = 0; j < N; ++j) {
            double v = 0.0;
            if (n < N)
                v = n >= j ? h[n - j] : 0.0;
            else if (n - N < S)
                v = g[static_cast<size_t>(N - 1 - j) * S + (n - N)];
            const float hi = head(v), lo = static_cast<float>(v - static_cast<double>(hi));
            const size_t half = static_cast<size_t>(j >> 5) * (HB / 2);
            put(half, n, j & 31, hi);
            put(HB + half, n, j & 31, lo);
        }
    for (int m = 0; m < N; ++m)
        for (int k = 0; k < S; ++k) {
            const double v = H[static_cast<size_t>(k) * N + m];
            const float hi = head(v), lo = static_cast<float>(v - static_cast<double>(hi));
            put(2 * HB, m, k, hi);
            put(2 * HB, m, 16 + k, lo);
        }
    std::vector<float> gt(static_cast<size_t>(S) * N);
    for (int k = 0; k < S; ++k)
        for (int j = 0; j < N; ++j) gt[static_cast<size_t>(k) * N + j] = static_cast<float>(g[static_cast<size_t>(N - 1 - j) * S + k]);
    if (cudaMalloc(&ps.d_tcimg, img.size()) != cudaSuccess ||
        cudaMalloc(&ps.d_gtail, gt.size() * sizeof(float)) != cudaSuccess)
        return SOS_ENOMEM;
    if (cudaMemcpy(ps.d_tcimg, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ps.d_gtail, gt.data(), gt.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return SOS_ECUDA;
    return SOS_OK;
}

int table_index(int N) {
    for (int i = 0; i < kNumN; ++i)
        if (kSupportedN[i] == N) return i;
    return -1;
}

// Default N of the cyclic-reduction paths: 64 measured fastest on GB300 at every order and length
// (N = 128 is built for b0-normalized filters only and is never the default).
int default_N(const sos_filter *, int64_t) { return 64; }

// The tag of every launch captured into a CUDA graph; eager launches never use it.
constexpr unsigned kCaptureEpoch = 0x3fffffffu;

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st == cudaStreamCaptureStatusActive;
}

// A launch being captured into a CUDA graph takes the filter's second ticket counter and the capture
// tag, and the graph resets both the counter and the launch's descriptors before the kernel, so that
// every replay starts afresh whatever ran before it; the eager launches' counter and tags are left
// as they are.  The workspace must already be large enough (no allocation while capturing).
sos_status capture_setup(sos_filter *f, cudaStream_t s, size_t desc_words, unsigned long long **ticket,
                         unsigned long long *base, unsigned *epoch) {
    if (!f->d_desc || desc_words > f->desc_groups * sosk::kMaxPass * 2) return SOS_EINVAL;
    if (cudaMemsetAsync(f->d_ticket + 1, 0, sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(f->d_desc, 0, desc_words * sizeof(unsigned long long), s) != cudaSuccess)
        return SOS_ECUDA;
    *ticket = f->d_ticket + 1;
    *base = 0;
    *epoch = kCaptureEpoch;
    return SOS_OK;
}

sos_status ensure_desc(sos_filter *f, long long G, cudaStream_t s) {
    if (static_cast<size_t>(G) <= f->desc_groups && f->d_desc) return SOS_OK;
    if (stream_capturing(s)) return SOS_EINVAL;  // no allocation inside a capture: run it once eagerly first
    size_t want = static_cast<size_t>(G);
    if (want < 1024) want = 1024;
    if (f->d_desc) {
        cudaStreamSynchronize(s);
        cudaFree(f->d_desc);
        f->d_desc = nullptr;
        f->desc_groups = 0;
    }
    const size_t bytes = want * sosk::kMaxPass * 2 * sizeof(unsigned long long);
    if (cudaMalloc(&f->d_desc, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SOS_ENOMEM;
    }
    if (cudaMemsetAsync(f->d_desc, 0, bytes, s) != cudaSuccess) return cuda_fail();
    f->desc_groups = want;
    f->epoch = 0;
    return SOS_OK;
}

unsigned next_epoch(sos_filter *f, cudaStream_t s) {
    f->epoch = f->epoch + 1;
    if (f->epoch >= kCaptureEpoch) {  // wrapped: clear stale tags so no old descriptor matches
        cudaMemsetAsync(f->d_desc, 0, f->desc_groups * sosk::kMaxPass * 2 * sizeof(unsigned long long), s);
        f->epoch = 1;
    }
    return f->epoch;
}



bool ranges_overlap(const void *a, const void *b, int64_t n) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    const uintptr_t bytes = static_cast<uintptr_t>(n) * sizeof(float);
    return x < y + bytes && y < x + bytes;
}

// Per-section carries: one decoupled lookback per section and thread block (sosfilt_dccr.cuh).
sos_status run_sections(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf,
                        cudaStream_t s) {
    if (stream_capturing(s)) return SOS_EINVAL;  // per-section carries are not captured into graphs
    int N = f->tuning.N ? f->tuning.N : default_N(f, n);
    if (N == 128 && !f->norm) N = 64;
    const int ti = table_index(N);
    if (ti < 0) return SOS_EINVAL;
    const NTables &t = f->tables[ti];
    const long long C = static_cast<long long>(N) * sosk::kL;
    const long long G = (n + C - 1) / C;
    sos_status st = ensure_desc(f, G, s);
    if (st != SOS_OK) return st;
    const long long grid = (G + sosk::kWarps - 1) / sosk::kWarps;
    for (int k0 = 0; k0 < f->K; k0 += sosk::kMaxPass) {
        const int kp = (f->K - k0) < sosk::kMaxPass ? (f->K - k0) : sosk::kMaxPass;
        if (!sosk::dccr_available(kp, N, f->norm, f->tuning.lookback_width)) return SOS_EINVAL;
    }
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    const float *src = x;
    for (int k0 = 0; k0 < f->K; k0 += sosk::kMaxPass) {
        const int kp = (f->K - k0) < sosk::kMaxPass ? (f->K - k0) : sosk::kMaxPass;
        sosk::PassParams p;
        std::memset(&p, 0, sizeof p);
        p.x = src;
        p.y = y;
        p.n = n;
        p.G = G;
        p.zi = zi ? zi + 2 * k0 : nullptr;
        p.zf = zf ? zf + 2 * k0 : nullptr;
        p.gain = (k0 == 0) ? static_cast<float>(f->gain) : 1.0f;
        p.desc = f->d_desc;
        p.ticket = f->d_ticket;
        p.ticket_base = f->ticket_base;
        p.epoch = next_epoch(f, s);
        p.lane_pow = t.d_lane_pow + static_cast<size_t>(k0) * 32;
        p.grp_pow = t.d_grp_pow + static_cast<size_t>(k0) * sosk::kGrpPowStride;
        p.cta_pow = t.d_cta_pow + static_cast<size_t>(k0) * sosk::kGrpPowStride;
        p.status = f->d_status;
        p.spin_budget = f->tuning.spin_budget_cycles ? f->tuning.spin_budget_cycles : kDefaultSpinBudget;
        p.aligned = aligned ? 1 : 0;
        p.n_sec = kp;
        p.trace = f->trace;
        p.trace_blocks = f->trace_blocks;
        for (int j = 0; j < kp; ++j) p.sec[j] = t.sec[k0 + j];
        // the gain multiplies the input only in the first pass (p.gain = 1 afterwards)
        cudaError_t e = sosk::launch_dccr(kp, N, f->norm, f->tuning.lookback_width, p, grid, s);
        if (e != cudaSuccess) return cuda_fail();
        f->ticket_base += static_cast<unsigned long long>(grid);
        src = y;
    }
    return SOS_OK;
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) n = 1;
    if (device >= 0 && device < 64) cached[device] = n;
    return n;
}

template <int K, int N>
sos_status launch_cascade_pass(sos_filter *f, CasPass &ps, const sosk::SecCoef *sec, const float *x, float *y,
                               long long n, long long G, long long n_tiles, long long grid, const float *zi,
                               float *zf, bool first, bool aligned, cudaStream_t s, bool dtcr = false) {
    static_assert(K >= 1 && K <= sosk::kMaxPass, "pass size");
    auto p = std::make_unique<sosk::CasParams<K, N>>();
    std::memset(p.get(), 0, sizeof(*p));
    p->x = x;
    p->y = y;
    p->n = n;
    p->G = G;
    p->n_tiles = n_tiles;
    p->zi = zi;
    p->zf = zf;
    p->gain = first ? static_cast<float>(f->gain) : 1.0f;
    p->desc = f->d_desc;
    const bool eager = !stream_capturing(s);
    if (eager) {
        p->ticket = f->d_ticket;
        p->ticket_base = f->ticket_base;
        p->epoch = next_epoch(f, s);
    } else {
        const sos_status cst = capture_setup(f, s, static_cast<size_t>(n_tiles) * 2 * K, &p->ticket,
                                             &p->ticket_base, &p->epoch);
        if (cst != SOS_OK) return cst;
    }
    p->status = f->d_status;
    p->spin_budget = f->tuning.spin_budget_cycles ? f->tuning.spin_budget_cycles : kDefaultSpinBudget;
    p->aligned = aligned ? 1 : 0;
    p->tab = ps.d_tab;
    p->trace = f->trace;
    p->trace_tiles = f->trace_blocks;
    for (int j = 0; j < K; ++j) p->sec[j] = sec[j];
    for (int j = 0; j < 2 * K; ++j)
        for (int m = 0; m < N; ++m) p->H[j][m] = ps.H[static_cast<size_t>(j) * N + m];
    if (zf) {
        const long long C = 32LL * N;
        const long long tp = n - 1 - (G - 1) * C;  // last real sample inside the last group
        if (ps.tail_p != tp) {
            ps.A_tail.assign(packed_floats(K), 0.f);
            pack_into(dpow(ps.M1, tp + 1), K, ps.A_tail.data());
            ps.tail_p = tp;
        }
        std::memcpy(p->A_tail, ps.A_tail.data(), sizeof(float) * packed_floats(K));
    }
    cudaError_t e;
    if constexpr (N == 64)
        e = dtcr ? sosk::launch_dtcr<K>(f->norm, *p, grid, s) : sosk::launch_cascade<K, N>(f->norm, *p, grid, s);
    else
        e = sosk::launch_cascade<K, N>(f->norm, *p, grid, s);
    if (e != cudaSuccess) return SOS_ECUDA;
    if (eager) f->ticket_base += static_cast<unsigned long long>(n_tiles + grid);
    return SOS_OK;
}

template <int N>
sos_status launch_cascade_any(int K, sos_filter *f, CasPass &ps, const sosk::SecCoef *sec, const float *x, float *y,
                              long long n, long long G, long long n_tiles, long long grid, const float *zi, float *zf,
                              bool first, bool aligned, cudaStream_t s, bool dtcr = false) {
    switch (K) {
#define SOSK_CASE(k) \
    case k: return launch_cascade_pass<k, N>(f, ps, sec, x, y, n, G, n_tiles, grid, zi, zf, first, aligned, s, dtcr);
        SOSK_CASE(1) SOSK_CASE(2) SOSK_CASE(3) SOSK_CASE(4) SOSK_CASE(5) SOSK_CASE(6) SOSK_CASE(7) SOSK_CASE(8)
#undef SOSK_CASE
        default: return SOS_EINVAL;
    }
}

// One carry per tile for the whole cascade (sosfilt_cascade.cuh), persistent grid.
sos_status run_cascade(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf,
                       cudaStream_t s, int N_choice = 0) {
    // default N from GB300 measurements on 2^28 samples (cascade carry): N = 64 for one section
    // (HBM-bound, fewer tiles per sample), N = 32 otherwise (more warps to hide the pass's latency)
    int N = f->tuning.N ? f->tuning.N : N_choice ? N_choice : (f->K == 1 ? 64 : 32);
    if (N != 32 && N != 64) return SOS_EINVAL;
    const int ci = (N == 32) ? 0 : 1;
    const int ti = table_index(N);
    const long long C = 32LL * N;
    const long long W = sosk::cascade_warps(N);
    const long long G = (n + C - 1) / C;
    const long long n_tiles = (G + W - 1) / W;
    sos_status st = ensure_desc(f, G, s);
    if (st != SOS_OK) return st;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    const float *src = x;
    for (auto &ps : f->cas[ci].passes) {
        const int bps = sosk::cascade_blocks_per_sm(ps.kp, N, f->norm);
        if (bps <= 0) return SOS_ECUDA;
        long long grid = static_cast<long long>(bps) * sm_count(f->device);
        if (grid > n_tiles) grid = n_tiles;
        if (N == 32)
            st = launch_cascade_any<32>(ps.kp, f, ps, &f->tables[ti].sec[ps.k0], src, y, n, G, n_tiles, grid,
                                        zi ? zi + 2 * ps.k0 : nullptr, zf ? zf + 2 * ps.k0 : nullptr, ps.k0 == 0,
                                        aligned, s);
        else
            st = launch_cascade_any<64>(ps.kp, f, ps, &f->tables[ti].sec[ps.k0], src, y, n, G, n_tiles, grid,
                                        zi ? zi + 2 * ps.k0 : nullptr, zf ? zf + 2 * ps.k0 : nullptr, ps.k0 == 0,
                                        aligned, s);
        if (st != SOS_OK) return st;
        src = y;
    }
    return SOS_OK;
}

// Double-thread-group cyclic reduction (sosfilt_dtcr.cuh): the cascade carry on the N = 64
// cyclic-reduction tables, two warps (one per parity) per group.
sos_status run_dtcr(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf, cudaStream_t s) {
    constexpr int N = 64;
    const int ti = table_index(N);
    const long long C = 32LL * N;
    const long long W = sosk::cascade_warps(N);
    const long long G = (n + C - 1) / C;
    const long long n_tiles = (G + W - 1) / W;
    sos_status st = ensure_desc(f, G, s);
    if (st != SOS_OK) return st;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    const float *src = x;
    for (auto &ps : f->cas[1].passes) {
        const int bps = sosk::dtcr_blocks_per_sm(ps.kp, f->norm);
        if (bps <= 0) return SOS_ECUDA;
        long long grid = static_cast<long long>(bps) * sm_count(f->device);
        if (grid > n_tiles) grid = n_tiles;
        st = launch_cascade_any<64>(ps.kp, f, ps, &f->tables[ti].sec[ps.k0], src, y, n, G, n_tiles, grid,
                                    zi ? zi + 2 * ps.k0 : nullptr, zf ? zf + 2 * ps.k0 : nullptr, ps.k0 == 0, aligned, s,
                                    true);
        if (st != SOS_OK) return st;
        src = y;
    }
    return SOS_OK;
}

// ---- skewed-pass PH kernel (sosfilt_lane.cuh)
template <int K, int N, int W, bool TC = false>
sos_status launch_lane_pass(sos_filter *f, LanePass &ps, const float *x, float *y, long long n, long long G,
                            long long n_tiles, long long grid, const float *zi, float *zf, bool first, bool aligned,
                            cudaStream_t s, const sosk::Scratch *sc = nullptr, unsigned sc_epoch = 0) {
    static_assert(K >= 1 && K <= sosk::kMaxPass, "pass size");
    // the parameter block lives on the stack (about 2 KB at K = 8): a run does no host allocation
    sosk::LaneParams<K> pb;
    std::memset(&pb, 0, sizeof(pb));
    sosk::LaneParams<K> *p = &pb;
    p->x = x;
    p->y = y;
    p->n = n;
    p->G = G;
    p->n_tiles = n_tiles;
    p->zi = zi;
    p->zf = zf;
    p->gain = first ? static_cast<float>(f->gain) : 1.0f;
    if (sc) {
        // caller-provided scratch (sos_filter_run_noalloc): its ticket counter starts from zero, and
        // the pass's descriptors are cleared, so that no descriptor of an earlier call can be taken
        // for this one whatever its tag (tags are never 0)
        if (cudaMemsetAsync(sc->ticket, 0, sizeof(unsigned long long), s) != cudaSuccess) return SOS_ECUDA;
        if (cudaMemsetAsync(sc->desc, 0, static_cast<size_t>(n_tiles) * 2 * 2 * K * sizeof(unsigned long long), s) !=
            cudaSuccess)
            return SOS_ECUDA;
        p->desc = sc->desc;
        p->ticket = sc->ticket;
        p->ticket_base = 0;
        p->epoch = sc_epoch;
    } else if (stream_capturing(s)) {
        p->desc = f->d_desc;
        const sos_status cst = capture_setup(f, s, static_cast<size_t>(n_tiles) * 2 * 2 * K, &p->ticket,
                                             &p->ticket_base, &p->epoch);
        if (cst != SOS_OK) return cst;
    } else {
        p->desc = f->d_desc;
        p->ticket = f->d_ticket;
        p->ticket_base = f->ticket_base;
        p->epoch = next_epoch(f, s);
    }
    const bool eager = !sc && p->ticket == f->d_ticket;
    p->status = f->d_status;
    p->spin_budget = f->tuning.spin_budget_cycles ? f->tuning.spin_budget_cycles : kDefaultSpinBudget;
    p->aligned = aligned ? 1 : 0;
    p->tab = ps.d_tab;
    p->trace = f->trace;
    p->trace_tiles = f->trace_blocks;
    for (int j = 0; j < K; ++j) p->sec[j] = ps.sec[j];
    std::memcpy(p->MX, ps.MX.data(), sizeof(float) * ps.MX.size());
    const long long C = 32LL * N;
    const int m_last = static_cast<int>((n - 1 - (G - 1) * C) % N);
    p->m_last = m_last;
    if (zf) std::memcpy(p->A_tail, &ps.Mm[static_cast<size_t>(m_last) * packed_floats(K)], sizeof(float) * packed_floats(K));
    cudaError_t e;
    if constexpr (TC)
        e = sosk::launch_tc<K>(*p, ps.d_tcimg, ps.d_gtail, grid, s);
    else
        e = sosk::launch_lane<K, N, W>(f->norm, *p, grid, s);
    if (e != cudaSuccess) return SOS_ECUDA;
    if (eager) f->ticket_base += static_cast<unsigned long long>(n_tiles + grid);
    return SOS_OK;
}

template <int N, int W, bool TC = false>
sos_status launch_lane_any(int K, sos_filter *f, LanePass &ps, const float *x, float *y, long long n, long long G,
                           long long n_tiles, long long grid, const float *zi, float *zf, bool first, bool aligned,
                           cudaStream_t s, const sosk::Scratch *sc = nullptr, unsigned sc_epoch = 0) {
    switch (K) {
#define SOSK_CASE(k) \
    case k:          \
        return launch_lane_pass<k, N, W, TC>(f, ps, x, y, n, G, n_tiles, grid, zi, zf, first, aligned, s, sc, sc_epoch);
        SOSK_CASE(1) SOSK_CASE(2) SOSK_CASE(3) SOSK_CASE(4) SOSK_CASE(5) SOSK_CASE(6) SOSK_CASE(7) SOSK_CASE(8)
#undef SOSK_CASE
        default: return SOS_EINVAL;
    }
}

// PH factorization with the skewed particular pass, one carry per tile for the whole cascade,
// persistent grid.
sos_status run_lane(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf, cudaStream_t s,
                    int N_choice = 0, int W_choice = 0) {
    const int N = f->tuning.N ? f->tuning.N : N_choice ? N_choice : 64;
    if (N != 32 && N != 64) return SOS_EINVAL;
    const int Wv = N == 32 ? sosk::kLaneW
                           : f->tuning.groups_per_cta ? f->tuning.groups_per_cta : W_choice ? W_choice : sosk::kLaneW;
    if (Wv != sosk::kLaneW && Wv != sosk::kLaneWide) return SOS_EINVAL;
    auto &passes = f->lane[N == 32 ? 0 : Wv == sosk::kLaneWide ? 2 : 1];
    const long long C = 32LL * N;
    const long long W = Wv;
    const long long G = (n + C - 1) / C;
    const long long n_tiles = (G + W - 1) / W;
    sos_status st = ensure_desc(f, G, s);
    if (st != SOS_OK) return st;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    const float *src = x;
    for (auto &ps : passes) {
        const int bps = sosk::lane_blocks_per_sm(ps.kp, N, Wv, f->norm);
        if (bps <= 0) return SOS_ECUDA;
        long long grid = static_cast<long long>(bps) * sm_count(f->device);
        if (grid > n_tiles) grid = n_tiles;
        const float *zp = zi ? zi + 2 * ps.k0 : nullptr;
        float *zq = zf ? zf + 2 * ps.k0 : nullptr;
        if (N == 32)
            st = launch_lane_any<32, sosk::kLaneW>(ps.kp, f, ps, src, y, n, G, n_tiles, grid, zp, zq, ps.k0 == 0,
                                                   aligned, s);
        else if (Wv == sosk::kLaneWide)
            st = launch_lane_any<64, sosk::kLaneWide>(ps.kp, f, ps, src, y, n, G, n_tiles, grid, zp, zq, ps.k0 == 0,
                                                      aligned, s);
        else
            st = launch_lane_any<64, sosk::kLaneW>(ps.kp, f, ps, src, y, n, G, n_tiles, grid, zp, zq, ps.k0 == 0,
                                                   aligned, s);
        if (st != SOS_OK) return st;
        src = y;
    }
    return SOS_OK;
}

// PH factorization on the tensor cores (sosfilt_tc.cuh): tiles of kTcGroups groups of 32 rows of 64
// samples.  Its TMA copies need 16-byte aligned signals of at least one full row; other signals run
// the skewed-pass PH kernel.
sos_status run_tc(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf, cudaStream_t s) {
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    if (!aligned || n < 64) return run_lane(f, x, y, n, zi, zf, s, 64, sosk::kLaneW);
    constexpr long long C = 32LL * 64, W = sosk::kTcGroups;
    const long long G = (n + C - 1) / C;
    const long long n_tiles = (G + W - 1) / W;
    sos_status st = ensure_desc(f, G, s);
    if (st != SOS_OK) return st;
    const float *src = x;
    for (auto &ps : f->lane[3]) {
        const int bps = sosk::tc_blocks_per_sm(ps.kp);
        if (bps <= 0) return SOS_ECUDA;
        long long grid = static_cast<long long>(bps) * sm_count(f->device);
        if (grid > n_tiles) grid = n_tiles;
        const float *zp = zi ? zi + 2 * ps.k0 : nullptr;
        float *zq = zf ? zf + 2 * ps.k0 : nullptr;
        st = launch_lane_any<64, sosk::kTcGroups, true>(ps.kp, f, ps, src, y, n, G, n_tiles, grid, zp, zq,
                                                        ps.k0 == 0, true, s);
        if (st != SOS_OK) return st;
        src = y;
    }
    return SOS_OK;
}

// Solver of a run: the tuning's choice; by default PH factorization with the skewed particular
// pass (faster than cyclic reduction at every order on GB300 at 2^28 samples: 227 vs 154 GS/s at
// order 16, 606 vs 540 at order 2), unless the tuning asks for what only cyclic reduction has (a
// carry scheme, a lookback width, N = 128).
int solver_of(const sos_filter *f) {
    const sos_tuning &t = f->tuning;
    if (t.solver) return t.solver;
    if (t.carry || t.lookback_width || t.N == 128) return SOS_SOLVER_CR;
    return SOS_SOLVER_PH;
}

// ---- autotuned launch choice (sos_autotune): per device, section count (1..8) and length bucket
constexpr int kTuneBuckets = 4;                       // n around 2^16, 2^20, 2^24, 2^28
constexpr int kTuneLog2[kTuneBuckets] = {16, 20, 24, 28};
constexpr int kTuneCand = 6;  // candidates: CR N = 32, CR N = 64, PH (7 groups), DTCR, PH (10 groups), TC
struct TuneTable {
    bool valid = false;
    unsigned char best[8][kTuneBuckets] = {};         // candidate index
    float gss[8][kTuneBuckets][kTuneCand] = {};       // measured GS/s
};
std::mutex g_tune_mu;
TuneTable g_tune[64];

// Autotuned tile geometry of batched runs (sos_autotune_batch): per device, section count and
// signal length bucket, geometry 0 (N = 64) or 1 (N = 32).
constexpr int kBatchTuneBuckets = 4;  // signal lengths around 2^12, 2^15, 2^18, 2^21
constexpr int kBatchTuneLog2[kBatchTuneBuckets] = {12, 15, 18, 21};
struct BatchTune {
    bool valid = false;
    unsigned char geom[8][kBatchTuneBuckets] = {};
    float gss[8][kBatchTuneBuckets][sosk::kBatchGeoms] = {};  // measured GS/s
};
BatchTune g_btune[64];

int batch_tune_bucket(int64_t n) {
    int b = 0;
    for (int i = 1; i < kBatchTuneBuckets; ++i)
        if (n >= (1LL << ((kBatchTuneLog2[i - 1] + kBatchTuneLog2[i]) / 2))) b = i;
    return b;
}

// The tile geometry of one batched signal: the filter's pinned geometry, else the device's autotuned
// choice for its section count and length (a copy taken once per call), else N = 64.
struct BatchGeomChoice {
    bool valid = false;
    unsigned char geom[8][kBatchTuneBuckets] = {};
};
BatchGeomChoice batch_geom_choice(int device) {
    BatchGeomChoice c;
    if (device < 0 || device >= 64) return c;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    c.valid = g_btune[device].valid;
    std::memcpy(c.geom, g_btune[device].geom, sizeof c.geom);
    return c;
}
int batch_geom_of(const BatchTmpl &bt, int K, int64_t n, const BatchGeomChoice &gc) {
    if (bt.geom >= 0) return bt.geom;
    if (!gc.valid) return 0;
    return gc.geom[(K > sosk::kMaxPass ? sosk::kMaxPass : K) - 1][batch_tune_bucket(n)];
}

void candidate(int c, int *solver, int *N, int *W) {
    *solver = (c == 2 || c == 4) ? SOS_SOLVER_PH : c == 3 ? SOS_SOLVER_DTCR : c == 5 ? SOS_SOLVER_TC : SOS_SOLVER_CR;
    *N = c == 0 ? 32 : 64;
    *W = c == 4 ? sosk::kLaneWide : c == 2 ? sosk::kLaneW : c == 5 ? sosk::kTcGroups : 0;
}

int tune_bucket(int64_t n) {
    int b = 0;
    for (int i = 1; i < kTuneBuckets; ++i)
        if (n >= (1LL << ((kTuneLog2[i - 1] + kTuneLog2[i]) / 2))) b = i;
    return b;
}

bool tuned_choice(int device, int K, int64_t n, int *solver, int *N, int *W) {
    if (device < 0 || device >= 64) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune[device].valid) return false;
    const int k = (K > sosk::kMaxPass ? sosk::kMaxPass : K) - 1;
    candidate(g_tune[device].best[k][tune_bucket(n)], solver, N, W);
    return true;
}

sos_status run_impl(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf, cudaStream_t s) {
    if (n < 0 || (n > 0 && (!x || !y))) return SOS_EINVAL;
    if (x != y && n > 0 && ranges_overlap(x, y, n)) return SOS_EINVAL;
    if (cudaSetDevice(f->device) != cudaSuccess) return cuda_fail();
    f->last_stream = s;
    if (n == 0) {
        if (zf) {
            cudaError_t e = zi ? cudaMemcpyAsync(zf, zi, sizeof(float) * 2 * f->K, cudaMemcpyDeviceToDevice, s)
                               : cudaMemsetAsync(zf, 0, sizeof(float) * 2 * f->K, s);
            if (e != cudaSuccess) return cuda_fail();
        }
        return SOS_OK;
    }
    const sos_tuning &t = f->tuning;
    if (!t.N && !t.carry && !t.solver && !t.lookback_width && !t.groups_per_cta) {
        // all defaults: the autotuned choice for this section count and length, if there is one
        int solver = 0, N = 0, W = 0;
        if (tuned_choice(f->device, f->K, n, &solver, &N, &W)) {
            if (solver == SOS_SOLVER_PH) return run_lane(f, x, y, n, zi, zf, s, N, W);
            if (solver == SOS_SOLVER_DTCR) return run_dtcr(f, x, y, n, zi, zf, s);
            if (solver == SOS_SOLVER_TC) return run_tc(f, x, y, n, zi, zf, s);
            return run_cascade(f, x, y, n, zi, zf, s, N);
        }
    }
    if (solver_of(f) == SOS_SOLVER_PH) return run_lane(f, x, y, n, zi, zf, s);
    if (solver_of(f) == SOS_SOLVER_DTCR) return run_dtcr(f, x, y, n, zi, zf, s);
    if (solver_of(f) == SOS_SOLVER_TC) return run_tc(f, x, y, n, zi, zf, s);
    if (t.carry == SOS_CARRY_SECTION) return run_sections(f, x, y, n, zi, zf, s);
    return run_cascade(f, x, y, n, zi, zf, s);
}

// ---- multi-signal runs (sosfilt_batch.cuh)
constexpr int kBatchSlots = 8;     // batches whose scratch may be in use on the device at once
constexpr int kBatchClasses = sosk::kBatchClassesMax;  // (geometry, K, b0-normalized): sosk::batch_class

// Scratch of one batch in flight: signal descriptors and the tile -> signal map (one upload from
// pinned staging), lookback descriptors and the ticket counters of its classes.
struct BatchSlot {
    std::mutex mu;  // held by the call using the slot: its staging, capacities and event
    unsigned char *d_up = nullptr, *h_up = nullptr;  // [descriptors][tile -> signal map]
    size_t up_cap = 0;
    unsigned long long *d_desc = nullptr;
    size_t desc_cap = 0;
    unsigned long long *d_ticket = nullptr;  // [kBatchClasses]
    cudaEvent_t done = nullptr;
    bool pending = false;
};

struct BatchCtx {
    int device = -1;
    std::mutex mu;
    BatchSlot slot[kBatchSlots];
    int next = 0;
    int *d_status = nullptr;
    unsigned epoch = 0;
};

BatchCtx *batch_ctx(int device) {
    static std::mutex mu;
    static BatchCtx *ctx[64] = {nullptr};
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ctx[device]) {
        BatchCtx *c = new (std::nothrow) BatchCtx();
        if (!c) return nullptr;
        c->device = device;
        bool ok = cudaMalloc(&c->d_status, sizeof(int)) == cudaSuccess &&
                  cudaMemset(c->d_status, 0, sizeof(int)) == cudaSuccess;
        for (int i = 0; ok && i < kBatchSlots; ++i) {
            BatchSlot &sl = c->slot[i];
            ok = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                 cudaMalloc(&sl.d_ticket, sizeof(unsigned long long) * kBatchClasses) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            return nullptr;  // leaked on failure; the device is unusable anyway
        }
        ctx[device] = c;
    }
    return ctx[device];
}

// The single batch kernel's parameters: one queue per class present (its signal descriptors, tile ->
// signal map, lookback descriptors and ticket counter), the grid, and each class's share of the
// grid to start on, in proportion to its work (samples per tile x tiles x (2 + K), the particular
// pass and correction growing with K).
sos_status batch_all_params(const long long *cls_sigs, const long long *cls_tiles, const long long *sig_off,
                            const long long *tile_off, const long long *desc_off, const sosk::BatchSig *d_sigs,
                            const int *d_tile_sig, unsigned long long *d_desc, unsigned long long *d_ticket,
                            unsigned epoch, int *d_status, int device, sosk::BatchAllParams &ap, long long &grid) {
    std::memset(&ap, 0, sizeof ap);
    double work[kBatchClasses] = {0.0}, total = 0.0;
    long long tiles = 0;
    int nc = 0;
    for (int c = 0; c < kBatchClasses; ++c) {
        if (cls_sigs[c] == 0) continue;
        ap.code[nc] = c;
        ap.q[nc] = sosk::BatchQueue{d_sigs + sig_off[c], d_tile_sig + tile_off[c], cls_tiles[c], d_desc + desc_off[c],
                                    d_ticket + c, 0ULL, epoch};
        work[nc] = static_cast<double>(cls_tiles[c]) * sosk::batch_geom_n(sosk::batch_class_geom(c)) *
                   (2 + sosk::batch_class_k(c));
        total += work[nc];
        tiles += cls_tiles[c];
        ++nc;
    }
    ap.n_classes = nc;
    ap.status = d_status;
    ap.spin_budget = kDefaultSpinBudget;
    const int bps = sosk::batch_all_blocks_per_sm();
    if (bps <= 0) return SOS_ECUDA;
    grid = static_cast<long long>(bps) * sm_count(device);
    if (grid > tiles) grid = tiles;
    // shares: at least one block per class while blocks last, the rest by work
    double acc = 0.0;
    ap.blk_off[0] = 0;
    for (int i = 0; i < nc; ++i) {
        acc += work[i];
        long long end = static_cast<long long>(acc / total * static_cast<double>(grid) + 0.5);
        if (end <= ap.blk_off[i]) end = ap.blk_off[i] + 1;
        if (end > grid) end = grid;
        ap.blk_off[i + 1] = static_cast<int>(end);
    }
    ap.blk_off[nc] = static_cast<int>(grid);
    return SOS_OK;
}

sos_status run_batch_impl(int n_signals, sos_filter *const *filters, const float *const *x, float *const *y,
                          const int64_t *n, const float *const *zi, float *const *zf, cudaStream_t s) {
    if (n_signals < 0) return SOS_EINVAL;
    if (n_signals == 0) return SOS_OK;
    if (!filters || !x || !y || !n) return SOS_EINVAL;
    constexpr long long W = sosk::kBatchW;
    // arguments, classes and sizes in one pass over the signals (the per-signal work of a call
    // reads only the front cache line of each filter)
    const int device = filters[0] ? filters[0]->device : -1;
    const BatchGeomChoice gc = batch_geom_choice(device);
    long long cls_sigs[kBatchClasses] = {0}, cls_tiles[kBatchClasses] = {0};
    bool any_other = false;  // zero-length signals or filters of more than kMaxPass sections
    for (int i = 0; i < n_signals; ++i) {
        const sos_filter *f = filters[i];
        if (!f || n[i] < 0 || (n[i] > 0 && (!x[i] || !y[i]))) return SOS_EINVAL;
        if (x[i] != y[i] && n[i] > 0 && ranges_overlap(x[i], y[i], n[i])) return SOS_EINVAL;
        if (f->device != device) return SOS_EINVAL;
        const BatchTmpl &bt = f->bt;
        if (n[i] == 0 || bt.cls < 0) {
            any_other = true;
            continue;
        }
        const int g = batch_geom_of(bt, sosk::batch_class_k(bt.cls), n[i], gc);
        const int c = bt.cls + 16 * g;
        const long long C = 32LL * sosk::batch_geom_n(g);
        cls_sigs[c] += 1;
        cls_tiles[c] += ((n[i] + C - 1) / C + W - 1) / W;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SOS_ECUDA;
    BatchCtx *ctx = batch_ctx(device);
    if (!ctx) return SOS_ENOMEM;

    for (int i = 0; any_other && i < n_signals; ++i) {
        sos_filter *f = filters[i];
        if (n[i] != 0 && f->bt.cls >= 0) continue;
        if (n[i] == 0) {
            if (zf && zf[i]) {
                const size_t b = sizeof(float) * 2 * f->K;
                cudaError_t e = (zi && zi[i]) ? cudaMemcpyAsync(zf[i], zi[i], b, cudaMemcpyDeviceToDevice, s)
                                              : cudaMemsetAsync(zf[i], 0, b, s);
                if (e != cudaSuccess) return SOS_ECUDA;
            }
            continue;
        }
        std::lock_guard<std::mutex> fl(f->mu);  // more than kMaxPass sections: filtered on its own
        sos_status st = run_impl(f, x[i], y[i], n[i], zi ? zi[i] : nullptr, zf ? zf[i] : nullptr, s);
        if (st != SOS_OK) return st;
    }
    long long sig_off[kBatchClasses + 1] = {0}, tile_off[kBatchClasses + 1] = {0}, desc_off[kBatchClasses + 1] = {0};
    int n_cls = 0;
    for (int c = 0; c < kBatchClasses; ++c) {
        sig_off[c + 1] = sig_off[c] + cls_sigs[c];
        tile_off[c + 1] = tile_off[c] + cls_tiles[c];
        desc_off[c + 1] = desc_off[c] + cls_tiles[c] * 4 * sosk::batch_class_k(c);  // [tiles][2][2K]
        if (cls_sigs[c]) ++n_cls;
    }
    if (sig_off[kBatchClasses] == 0) return SOS_OK;

    // a scratch slot and the launch's epoch under the context's lock; the slot's own lock then covers
    // its use, so that calls from several threads plan and launch on different slots at once
    BatchSlot *slp = nullptr;
    unsigned epoch = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        slp = &ctx->slot[ctx->next];
        ctx->next = (ctx->next + 1) % kBatchSlots;
        ctx->epoch = (ctx->epoch + 1) & 0x3fffffffu;
        if (ctx->epoch == 0) {
            // wrapped (once in 2^30 calls): clear stale tags of every slot's descriptors, with every
            // slot held and the device idle
            std::unique_lock<std::mutex> held[kBatchSlots];
            for (int k = 0; k < kBatchSlots; ++k) held[k] = std::unique_lock<std::mutex>(ctx->slot[k].mu);
            if (cudaDeviceSynchronize() != cudaSuccess) return SOS_ECUDA;
            for (auto &o : ctx->slot)
                if (o.d_desc && cudaMemset(o.d_desc, 0, o.desc_cap * sizeof(unsigned long long)) != cudaSuccess)
                    return SOS_ECUDA;
            ctx->epoch = 1;
        }
        epoch = ctx->epoch;
    }
    BatchSlot &sl = *slp;
    std::lock_guard<std::mutex> slk(sl.mu);
    // the slot is free once its previous batch has completed on the device
    if (sl.pending && cudaEventSynchronize(sl.done) != cudaSuccess) return SOS_ECUDA;
    sl.pending = false;
    const size_t sig_bytes = sizeof(sosk::BatchSig) * sig_off[kBatchClasses];
    const size_t up_bytes = sig_bytes + sizeof(int) * tile_off[kBatchClasses];
    if (up_bytes > sl.up_cap) {
        size_t cap = sl.up_cap ? sl.up_cap : 1 << 16;
        while (cap < up_bytes) cap *= 2;
        if (sl.d_up) cudaFree(sl.d_up);
        if (sl.h_up) cudaFreeHost(sl.h_up);
        sl.d_up = sl.h_up = nullptr;
        sl.up_cap = 0;
        if (cudaMalloc(&sl.d_up, cap) != cudaSuccess || cudaMallocHost(&sl.h_up, cap) != cudaSuccess) {
            cudaGetLastError();
            return SOS_ENOMEM;
        }
        sl.up_cap = cap;
    }
    if (static_cast<size_t>(desc_off[kBatchClasses]) > sl.desc_cap) {
        if (sl.d_desc) {
            cudaFree(sl.d_desc);
            sl.d_desc = nullptr;
            sl.desc_cap = 0;
        }
        const size_t want = static_cast<size_t>(desc_off[kBatchClasses]) * 2;
        if (cudaMalloc(&sl.d_desc, want * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return SOS_ENOMEM;
        }
        if (cudaMemsetAsync(sl.d_desc, 0, want * sizeof(unsigned long long), s) != cudaSuccess) return SOS_ECUDA;
        sl.desc_cap = want;
    }
    sosk::BatchSig *h_sigs = reinterpret_cast<sosk::BatchSig *>(sl.h_up);
    int *h_tile_sig = reinterpret_cast<int *>(sl.h_up + sig_bytes);
    const sosk::BatchSig *d_sigs = reinterpret_cast<const sosk::BatchSig *>(sl.d_up);
    const int *d_tile_sig = reinterpret_cast<const int *>(sl.d_up + sig_bytes);

    // descriptors and the tile -> signal map, class by class
    long long fill_sig[kBatchClasses], fill_tile[kBatchClasses];
    for (int c = 0; c < kBatchClasses; ++c) {
        fill_sig[c] = sig_off[c];
        fill_tile[c] = tile_off[c];
    }
    for (int i = 0; i < n_signals; ++i) {
        const BatchTmpl &bt = filters[i]->bt;  // the batch kernel's tables, read only
        if (bt.cls < 0 || n[i] == 0) continue;
        const int g = batch_geom_of(bt, sosk::batch_class_k(bt.cls), n[i], gc);
        const int c = bt.cls + 16 * g;
        const long long C = 32LL * sosk::batch_geom_n(g);
        const long long G = (n[i] + C - 1) / C;
        const long long nt = (G + W - 1) / W;
        const long long si = fill_sig[c]++;
        sosk::BatchSig &b = h_sigs[si];
        b.x = x[i];
        b.y = y[i];
        b.n = n[i];
        b.G = G;
        b.tile0 = fill_tile[c] - tile_off[c];
        b.zi = zi ? zi[i] : nullptr;
        b.zf = zf ? zf[i] : nullptr;
        b.sec = bt.sec[g];
        b.MX = bt.MX[g];
        b.tab = bt.tab[g];
        b.Mm = bt.Mm;
        b.gain = bt.gain;
        b.aligned = ((reinterpret_cast<uintptr_t>(x[i]) | reinterpret_cast<uintptr_t>(y[i])) % 16 == 0) ? 1 : 0;
        const int local = static_cast<int>(si - sig_off[c]);
        int *tm = h_tile_sig + fill_tile[c];
        for (long long t = 0; t < nt; ++t) tm[t] = local;
        fill_tile[c] += nt;
    }
    if (cudaMemcpyAsync(sl.d_up, sl.h_up, up_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(sl.d_ticket, 0, sizeof(unsigned long long) * kBatchClasses, s) != cudaSuccess)
        return SOS_ECUDA;

    // one persistent launch over every class (sos_batch_all_kernel)
    sosk::BatchAllParams ap;
    long long grid = 0;
    sos_status pst = batch_all_params(cls_sigs, cls_tiles, sig_off, tile_off, desc_off, d_sigs, d_tile_sig, sl.d_desc,
                                      sl.d_ticket, epoch, ctx->d_status, device, ap, grid);
    if (pst != SOS_OK) return pst;
    if (sosk::launch_batch_all(ap, grid, s) != cudaSuccess) return SOS_ECUDA;
    if (cudaEventRecord(sl.done, s) != cudaSuccess) return SOS_ECUDA;
    sl.pending = true;
    return SOS_OK;
}

}  // namespace

// A prepared batch (sos_batch_plan_*): descriptors uploaded once, launches enqueue no host work.
struct sos_batch_plan {
    int device = -1;
    int n_cls = 0;
    long long tiles[kBatchClasses] = {};
    const sosk::BatchSig *sigs[kBatchClasses] = {};
    const int *tile_sig[kBatchClasses] = {};
    unsigned long long *desc[kBatchClasses] = {};
    unsigned char *d_up = nullptr;            // descriptors and tile -> signal maps
    unsigned long long *d_desc = nullptr;     // lookback descriptors of every class
    size_t desc_words = 0;
    unsigned long long *d_ticket = nullptr;   // [kBatchClasses]
    int *d_status = nullptr;
};

namespace {

void plan_free(sos_batch_plan *p) {
    if (!p) return;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    if (p->d_up) cudaFree(p->d_up);
    if (p->d_desc) cudaFree(p->d_desc);
    if (p->d_ticket) cudaFree(p->d_ticket);
    if (p->d_status) cudaFree(p->d_status);
    delete p;
}

sos_status plan_create(int n_signals, sos_filter *const *filters, const float *const *x, float *const *y,
                       const int64_t *n, const float *const *zi, float *const *zf, sos_batch_plan **out) {
    if (!out || n_signals <= 0 || !filters || !x || !y || !n) return SOS_EINVAL;
    *out = nullptr;
    constexpr long long W = sosk::kBatchW;
    int device = filters[0] ? filters[0]->device : -1;
    const BatchGeomChoice gc = batch_geom_choice(device);
    long long cls_sigs[kBatchClasses] = {0}, cls_tiles[kBatchClasses] = {0};
    std::vector<int> cls(n_signals);
    for (int i = 0; i < n_signals; ++i) {
        sos_filter *f = filters[i];
        if (!f || f->device != device || n[i] <= 0 || !x[i] || !y[i] || f->K > sosk::kMaxPass) return SOS_EINVAL;
        if (x[i] != y[i] && ranges_overlap(x[i], y[i], n[i])) return SOS_EINVAL;
        const int g = batch_geom_of(f->bt, f->K, n[i], gc);
        const int c = sosk::batch_class(g, f->K, f->norm);
        cls[i] = c;
        cls_sigs[c] += 1;
        const long long C = 32LL * sosk::batch_geom_n(g);
        const long long G = (n[i] + C - 1) / C;
        cls_tiles[c] += (G + W - 1) / W;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SOS_ECUDA;
    long long sig_off[kBatchClasses + 1] = {0}, tile_off[kBatchClasses + 1] = {0}, desc_off[kBatchClasses + 1] = {0};
    for (int c = 0; c < kBatchClasses; ++c) {
        sig_off[c + 1] = sig_off[c] + cls_sigs[c];
        tile_off[c + 1] = tile_off[c] + cls_tiles[c];
        desc_off[c + 1] = desc_off[c] + cls_tiles[c] * 4 * sosk::batch_class_k(c);  // [tiles][2][2K]
    }
    const size_t sig_bytes = sizeof(sosk::BatchSig) * sig_off[kBatchClasses];
    const size_t up_bytes = sig_bytes + sizeof(int) * tile_off[kBatchClasses];
    std::vector<unsigned char> up(up_bytes);
    sosk::BatchSig *h_sigs = reinterpret_cast<sosk::BatchSig *>(up.data());
    int *h_tile_sig = reinterpret_cast<int *>(up.data() + sig_bytes);
    long long fill_sig[kBatchClasses], fill_tile[kBatchClasses];
    for (int c = 0; c < kBatchClasses; ++c) {
        fill_sig[c] = sig_off[c];
        fill_tile[c] = tile_off[c];
    }
    for (int i = 0; i < n_signals; ++i) {
        const int c = cls[i];
        const int g = sosk::batch_class_geom(c);
        sos_filter *f = filters[i];
        const BatchTmpl &bt = f->bt;  // the batch kernel's tables for the signal's geometry (read only)
        const long long C = 32LL * sosk::batch_geom_n(g);
        const long long G = (n[i] + C - 1) / C;
        const long long nt = (G + W - 1) / W;
        const long long si = fill_sig[c]++;
        sosk::BatchSig &b = h_sigs[si];
        b.x = x[i];
        b.y = y[i];
        b.n = n[i];
        b.G = G;
        b.tile0 = fill_tile[c] - tile_off[c];
        b.zi = zi ? zi[i] : nullptr;
        b.zf = zf ? zf[i] : nullptr;
        b.sec = bt.sec[g];
        b.MX = bt.MX[g];
        b.tab = bt.tab[g];
        b.Mm = bt.Mm;
        b.gain = bt.gain;
        b.aligned = (reinterpret_cast<uintptr_t>(x[i]) % 16 == 0 && reinterpret_cast<uintptr_t>(y[i]) % 16 == 0) ? 1 : 0;
        const int local = static_cast<int>(si - sig_off[c]);
        for (long long t = 0; t < nt; ++t) h_tile_sig[fill_tile[c]++] = local;
    }
    sos_batch_plan *p = new (std::nothrow) sos_batch_plan();
    if (!p) return SOS_ENOMEM;
    p->device = device;
    p->desc_words = static_cast<size_t>(desc_off[kBatchClasses]);
    bool ok = cudaMalloc(&p->d_up, up_bytes) == cudaSuccess &&
              cudaMalloc(&p->d_desc, sizeof(unsigned long long) * (p->desc_words + 1)) == cudaSuccess &&
              cudaMalloc(&p->d_ticket, sizeof(unsigned long long) * kBatchClasses) == cudaSuccess &&
              cudaMalloc(&p->d_status, sizeof(int)) == cudaSuccess &&
              cudaMemcpy(p->d_up, up.data(), up_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(p->d_status, 0, sizeof(int)) == cudaSuccess && sosk::batch_all_blocks_per_sm() > 0;
    for (int c = 0; ok && c < kBatchClasses; ++c) {
        if (!cls_sigs[c]) continue;
        p->tiles[c] = cls_tiles[c];
        p->sigs[c] = reinterpret_cast<const sosk::BatchSig *>(p->d_up) + sig_off[c];
        p->tile_sig[c] = reinterpret_cast<const int *>(p->d_up + sig_bytes) + tile_off[c];
        p->desc[c] = p->d_desc + desc_off[c];
        p->n_cls += 1;
    }
    if (!ok) {
        cudaGetLastError();
        plan_free(p);
        return SOS_ENOMEM;
    }
    *out = p;
    return SOS_OK;
}

// Status of a filter's finished work.  A launch that gave up on a wait (SOS_ETIMEOUT) consumed fewer
// tickets than the host counted, so once reported the status word and the ticket counter start over
// and later runs are valid again.
sos_status take_filter_status(sos_filter *f) {
    int h = 0;
    if (cudaMemcpy(&h, f->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
    if (!(h & sosk::kDevErrTimeout)) return SOS_OK;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemset(f->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(f->d_ticket, 0, sizeof(unsigned long long)) != cudaSuccess)
        return SOS_ECUDA;
    f->ticket_base = 0;
    return SOS_ETIMEOUT;
}

// Sticky device status of the batch context of a device (SOS_ETIMEOUT after a lookback timeout).
sos_status batch_status(int device) {
    BatchCtx *ctx = batch_ctx(device);
    if (!ctx) return SOS_ENOMEM;
    int h = 0;
    if (cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
    return (h & sosk::kDevErrTimeout) ? SOS_ETIMEOUT : SOS_OK;
}

}  // namespace

namespace sosk {
// Cascade-carry run whose lookback descriptors and ticket counter live in caller-provided device
// memory (sc); every pass takes a fresh epoch from next_epoch.  Allocates nothing.
int filter_device(const sos_filter *f) { return f->device; }

sos_status run_lane_scratch(sos_filter *f, const float *x, float *y, int64_t n, const float *zi, float *zf,
                            cudaStream_t s, const Scratch &sc, unsigned (*next_epoch)(int, cudaStream_t)) {
    if (!f || n < 0 || (n > 0 && (!x || !y))) return SOS_EINVAL;
    if (x != y && n > 0 && ranges_overlap(x, y, n)) return SOS_EINVAL;
    if (cudaSetDevice(f->device) != cudaSuccess) return SOS_ECUDA;
    f->last_stream = s;
    if (n == 0) {
        if (zf) {
            cudaError_t e = zi ? cudaMemcpyAsync(zf, zi, sizeof(float) * 2 * f->K, cudaMemcpyDeviceToDevice, s)
                               : cudaMemsetAsync(zf, 0, sizeof(float) * 2 * f->K, s);
            if (e != cudaSuccess) return SOS_ECUDA;
        }
        return SOS_OK;
    }
    // the default solver (PH factorization, N = 64) with the descriptors and ticket counter in sc
    constexpr int N = 64;
    const long long C = 32LL * N;
    const long long W = kLaneW;
    const long long G = (n + C - 1) / C;
    const long long n_tiles = (G + W - 1) / W;
    if (static_cast<size_t>(n_tiles) * 2 * 2 * kMaxPass > sc.desc_words) return SOS_EBUDGET;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
    const float *src = x;
    for (auto &ps : f->lane[1]) {
        const int bps = lane_blocks_per_sm(ps.kp, N, kLaneW, f->norm);
        if (bps <= 0) return SOS_ECUDA;
        long long grid = static_cast<long long>(bps) * sm_count(f->device);
        if (grid > n_tiles) grid = n_tiles;
        const unsigned epoch = next_epoch(f->device, s);
        const sos_status st = launch_lane_any<64, kLaneW>(ps.kp, f, ps, src, y, n, G, n_tiles, grid,
                                                  zi ? zi + 2 * ps.k0 : nullptr, zf ? zf + 2 * ps.k0 : nullptr,
                                                  ps.k0 == 0, aligned, s, &sc, epoch);
        if (st != SOS_OK) return st;
        src = y;
    }
    return SOS_OK;
}
}  // namespace sosk

extern "C" {

const char *sos_status_string(sos_status s) {
    switch (s) {
        case SOS_OK: return "SOS_OK";
        case SOS_EINVAL: return "SOS_EINVAL: invalid argument";
        case SOS_ENOMEM: return "SOS_ENOMEM: allocation failed";
        case SOS_ECUDA: return "SOS_ECUDA: CUDA runtime error";
        case SOS_ETIMEOUT: return "SOS_ETIMEOUT: lookback wait exceeded its budget";
        case SOS_EUNSTABLE: return "SOS_EUNSTABLE: unstable or non-finite section";
        case SOS_EBUDGET: return "SOS_EBUDGET: request exceeds the memory budget";
    }
    return "unknown sos_status";
}

sos_status sos_filter_create(int n_sections, const double *sos, const float *zi, const sos_tuning *t,
                             sos_filter **out) {
    if (!out) return SOS_EINVAL;
    *out = nullptr;
    if (!sos || n_sections < 1 || n_sections > 64) return SOS_EINVAL;
    if (t) {
        if (t->N && t->N != 32 && t->N != 64 && t->N != 128) return SOS_EINVAL;
        if (t->L && t->L != sosk::kL) return SOS_EINVAL;
        if (t->threads_per_group && t->threads_per_group != sosk::kL) return SOS_EINVAL;
        // groups per tile: chosen by the library (0), or for the PH solver 7, or 10 at N = 64
        if (t->groups_per_cta && t->groups_per_cta != sosk::kLaneW && t->groups_per_cta != sosk::kLaneWide)
            return SOS_EINVAL;
        if (t->groups_per_cta) {
            const bool ph = t->solver == SOS_SOLVER_PH ||
                            (t->solver == SOS_SOLVER_DEFAULT && !t->carry && !t->lookback_width && t->N != 128);
            if (!ph || (t->groups_per_cta == sosk::kLaneWide && t->N == 32)) return SOS_EINVAL;
        }
        if (t->fp64_carry) return SOS_EINVAL;
        if (t->spin_budget_cycles < 0) return SOS_EINVAL;
        if (t->carry != SOS_CARRY_DEFAULT && t->carry != SOS_CARRY_CASCADE && t->carry != SOS_CARRY_SECTION)
            return SOS_EINVAL;
        if ((t->carry == SOS_CARRY_DEFAULT || t->carry == SOS_CARRY_CASCADE) && t->N && t->N != 32 && t->N != 64)
            return SOS_EINVAL;
        const int lw = t->lookback_width;
        if (lw != 0 && lw != 1 && lw != 2 && lw != 4 && lw != 8 && lw != 16) return SOS_EINVAL;
        if (t->solver != SOS_SOLVER_DEFAULT && t->solver != SOS_SOLVER_CR && t->solver != SOS_SOLVER_PH &&
            t->solver != SOS_SOLVER_DTCR && t->solver != SOS_SOLVER_TC)
            return SOS_EINVAL;
        if (t->solver == SOS_SOLVER_TC &&
            ((t->N && t->N != 64) || t->carry == SOS_CARRY_SECTION || t->lookback_width || t->groups_per_cta))
            return SOS_EINVAL;
        if (t->solver == SOS_SOLVER_DTCR &&
            ((t->N && t->N != 64) || t->carry == SOS_CARRY_SECTION || t->lookback_width))
            return SOS_EINVAL;
        if (t->solver == SOS_SOLVER_PH &&
            ((t->N && t->N != 32 && t->N != 64) || t->carry == SOS_CARRY_SECTION || t->lookback_width))
            return SOS_EINVAL;
        if (t->deterministic != 0 && t->deterministic != 1) return SOS_EINVAL;
        if (t->deterministic && (t->solver == SOS_SOLVER_CR || t->solver == SOS_SOLVER_DTCR || t->carry ||
                                 t->lookback_width || t->N == 128))
            return SOS_EINVAL;
    }
    for (int k = 0; k < n_sections; ++k) {
        for (int j = 0; j < 5; ++j)
            if (!std::isfinite(sos[5 * k + j])) return SOS_EUNSTABLE;
        if (!section_stable(sos[5 * k + 3], sos[5 * k + 4])) return SOS_EUNSTABLE;
    }
    sos_filter *f = new (std::nothrow) sos_filter();
    if (!f) return SOS_ENOMEM;
    f->K = n_sections;
    f->sos.assign(sos, sos + 5 * n_sections);
    if (t) f->tuning = *t;
    if (cudaGetDevice(&f->device) != cudaSuccess) {
        delete f;
        return SOS_ECUDA;
    }
    // b0 normalization (Eq. 1 splits b0 into a common gain): legal when every b0 != 0 and
    // the gain and the per-section state scales stay far inside the float32 range.
    bool norm = true;
    double gain = 1.0;
    for (int k = 0; k < n_sections; ++k) {
        if (sos[5 * k] == 0.0) norm = false;
        gain *= sos[5 * k];
    }
    f->zscale.assign(n_sections, 1.0);
    if (norm) {
        for (int k = 0; k < n_sections; ++k) {
            double z = 1.0;
            for (int j = k + 1; j < n_sections; ++j) z *= sos[5 * j];
            f->zscale[k] = z;
            if (!(std::fabs(z) > 1e-30 && std::fabs(z) < 1e30)) norm = false;
        }
        if (!(std::fabs(gain) > 1e-30 && std::fabs(gain) < 1e30)) norm = false;
    }
    if (!norm) f->zscale.assign(n_sections, 1.0);
    f->norm = norm;
    f->gain = norm ? gain : 1.0;

    sos_status st = SOS_OK;
    for (int i = 0; i < kNumN && st == SOS_OK; ++i) {
        std::vector<float4> lp, gp, cp;
        build_tables(f, kSupportedN[i], f->tables[i], lp, gp, cp);
        if (cudaMalloc(&f->tables[i].d_lane_pow, lp.size() * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&f->tables[i].d_grp_pow, gp.size() * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&f->tables[i].d_cta_pow, cp.size() * sizeof(float4)) != cudaSuccess) {
            st = SOS_ENOMEM;
            break;
        }
        if (cudaMemcpy(f->tables[i].d_lane_pow, lp.data(), lp.size() * sizeof(float4), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(f->tables[i].d_grp_pow, gp.data(), gp.size() * sizeof(float4), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(f->tables[i].d_cta_pow, cp.data(), cp.size() * sizeof(float4), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            st = SOS_ECUDA;
    }
    for (int i = 0; i < 2 && st == SOS_OK; ++i) st = build_cascade(f, i == 0 ? 32 : 64, f->cas[i]);
    for (int i = 0; i < 4 && st == SOS_OK; ++i)
        st = build_lane(f, i == 0 ? 32 : 64, i == 2 ? sosk::kLaneWide : i == 3 ? sosk::kTcGroups : sosk::kLaneW,
                        f->lane[i]);
    for (size_t i = 0; i < f->lane[3].size() && st == SOS_OK; ++i) st = build_tc(f, f->lane[3][i]);
    if (st == SOS_OK) {
        for (int g = 0; g < sosk::kBatchGeoms; ++g) {
            const LanePass &ps = f->lane[g == 0 ? 1 : 0][0];  // (64, kBatchW) and (32, kBatchW)
            f->bt.sec[g] = ps.d_sec;
            f->bt.MX[g] = ps.d_MX;
            f->bt.tab[g] = ps.d_tab;
        }
        f->bt.Mm = f->lane[1][0].d_Mm;
        f->bt.gain = static_cast<float>(f->gain);
        f->bt.cls = static_cast<short>(f->K > sosk::kMaxPass ? -1 : sosk::batch_class(0, f->K, f->norm));
        f->bt.geom = static_cast<signed char>(f->tuning.N == sosk::kBatchNs ? 1 : f->tuning.N ? 0 : -1);
    }
    if (st == SOS_OK) {
        if (cudaMalloc(&f->d_ticket, 2 * sizeof(unsigned long long)) != cudaSuccess ||  // eager, captured
            cudaMalloc(&f->d_status, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&f->d_state, sizeof(float) * 2 * n_sections) != cudaSuccess)
            st = SOS_ENOMEM;
    }
    if (st == SOS_OK) {
        if (cudaMemset(f->d_ticket, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(f->d_status, 0, sizeof(int)) != cudaSuccess)
            st = SOS_ECUDA;
        std::vector<float> z(2 * n_sections, 0.f);
        if (zi) std::memcpy(z.data(), zi, sizeof(float) * 2 * n_sections);
        if (st == SOS_OK &&
            cudaMemcpy(f->d_state, z.data(), sizeof(float) * 2 * n_sections, cudaMemcpyHostToDevice) != cudaSuccess)
            st = SOS_ECUDA;
    }
    if (st != SOS_OK) {
        cudaGetLastError();
        sos_filter_destroy(f);
        return st;
    }
    *out = f;
    return SOS_OK;
}

sos_status sos_filter_destroy(sos_filter *f) {
    if (!f) return SOS_OK;
    cudaSetDevice(f->device);
    // the device, not the last stream: that stream may be gone, and batched runs may still read this
    // filter's tables on library streams
    cudaDeviceSynchronize();
    for (auto &t : f->tables) {
        if (t.d_lane_pow) cudaFree(t.d_lane_pow);
        if (t.d_grp_pow) cudaFree(t.d_grp_pow);
        if (t.d_cta_pow) cudaFree(t.d_cta_pow);
    }
    for (auto &ct : f->cas)
        for (auto &ps : ct.passes) {
            if (ps.d_tab) cudaFree(ps.d_tab);
        }
    for (auto &v : f->lane)
        for (auto &ps : v) {
            if (ps.d_tab) cudaFree(ps.d_tab);
            if (ps.d_sec) cudaFree(ps.d_sec);
            if (ps.d_MX) cudaFree(ps.d_MX);
            if (ps.d_Mm) cudaFree(ps.d_Mm);
            if (ps.d_tcimg) cudaFree(ps.d_tcimg);
            if (ps.d_gtail) cudaFree(ps.d_gtail);
        }
    if (f->d_desc) cudaFree(f->d_desc);
    if (f->d_ticket) cudaFree(f->d_ticket);
    if (f->d_status) cudaFree(f->d_status);
    if (f->d_state) cudaFree(f->d_state);
    for (int i = 0; i < 3; ++i) {
        if (f->hs[i]) cudaStreamDestroy(f->hs[i]);
        if (f->ev_in[i]) cudaEventDestroy(f->ev_in[i]);
        if (f->ev_done[i]) cudaEventDestroy(f->ev_done[i]);
        if (f->ev_out[i]) cudaEventDestroy(f->ev_out[i]);
        if (f->hbuf[i]) cudaFree(f->hbuf[i]);
    }
    if (f->d_hstate) cudaFree(f->d_hstate);
    delete f;
    return SOS_OK;
}

sos_status sos_filter_run(sos_filter *f, const float *x_dev, float *y_dev, int64_t n, const float *zi_dev,
                          float *zf_dev, void *stream) {
    if (!f) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    return run_impl(f, x_dev, y_dev, n, zi_dev, zf_dev, static_cast<cudaStream_t>(stream));
}

namespace {
// Streams, events and the state buffer of the host-buffer paths, created on first use.
sos_status ensure_host_pipeline(sos_filter *f) {
    if (f->hs[0]) return SOS_OK;
    for (int i = 0; i < 3; ++i) {
        if (cudaStreamCreateWithFlags(&f->hs[i], cudaStreamNonBlocking) != cudaSuccess) return SOS_ECUDA;
        if (cudaEventCreateWithFlags(&f->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&f->ev_done[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&f->ev_out[i], cudaEventDisableTiming) != cudaSuccess)
            return SOS_ECUDA;
    }
    if (cudaMalloc(&f->d_hstate, sizeof(float) * 2 * f->K) != cudaSuccess) return SOS_ENOMEM;
    return SOS_OK;
}

// The kernels read x_host and write y_host in place, through the buffers' device mappings (pinned or
// registered host memory): no staging copies, the signal crosses the CPU-GPU link once each way.
sos_status run_host_direct(sos_filter *f, const float *x_host, float *y_host, int64_t n, const float *zi_host,
                           float *zf_host) {
    void *dx = nullptr, *dy = nullptr;
    if (n > 0) {
        if (cudaHostGetDevicePointer(&dx, const_cast<float *>(x_host), 0) != cudaSuccess ||
            cudaHostGetDevicePointer(&dy, y_host, 0) != cudaSuccess || !dx || !dy) {
            cudaGetLastError();
            return SOS_EINVAL;  // not device-accessible host memory
        }
    }
    cudaStream_t sc = f->hs[1];
    const size_t zbytes = sizeof(float) * 2 * f->K;
    cudaError_t e = zi_host ? cudaMemcpyAsync(f->d_hstate, zi_host, zbytes, cudaMemcpyHostToDevice, sc)
                            : cudaMemsetAsync(f->d_hstate, 0, zbytes, sc);
    if (e != cudaSuccess) return SOS_ECUDA;
    const sos_status st = run_impl(f, static_cast<const float *>(dx), static_cast<float *>(dy), n, f->d_hstate,
                                   f->d_hstate, sc);
    if (st != SOS_OK) return st;
    if (zf_host && cudaMemcpyAsync(zf_host, f->d_hstate, zbytes, cudaMemcpyDeviceToHost, sc) != cudaSuccess)
        return SOS_ECUDA;
    if (cudaStreamSynchronize(sc) != cudaSuccess) return SOS_ECUDA;
    f->last_stream = sc;
    return take_filter_status(f);
}
}  // namespace

sos_status sos_filter_run_host(sos_filter *f, const float *x_host, float *y_host, int64_t n, const float *zi_host,
                               float *zf_host, int64_t chunk_samples) {
    if (!f || n < 0 || chunk_samples < SOS_HOST_DIRECT || (n > 0 && (!x_host || !y_host))) return SOS_EINVAL;
    if (x_host != y_host && n > 0 && ranges_overlap(x_host, y_host, n)) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    if (cudaSetDevice(f->device) != cudaSuccess) return SOS_ECUDA;
    sos_status pst = ensure_host_pipeline(f);
    if (pst != SOS_OK) return pst;
    if (chunk_samples == SOS_HOST_DIRECT) return run_host_direct(f, x_host, y_host, n, zi_host, zf_host);
    const long long chunk = chunk_samples ? chunk_samples : (1LL << 24);
    if (f->hbuf_samples < chunk) {
        for (int i = 0; i < 3; ++i) {
            if (f->hbuf[i]) cudaFree(f->hbuf[i]);
            f->hbuf[i] = nullptr;
        }
        f->hbuf_samples = 0;
        for (int i = 0; i < 3; ++i)
            if (cudaMalloc(&f->hbuf[i], sizeof(float) * chunk) != cudaSuccess) return SOS_ENOMEM;
        f->hbuf_samples = chunk;
    }
    cudaStream_t sin = f->hs[0], sc = f->hs[1], sout = f->hs[2];
    const size_t zbytes = sizeof(float) * 2 * f->K;
    cudaError_t e = zi_host ? cudaMemcpyAsync(f->d_hstate, zi_host, zbytes, cudaMemcpyHostToDevice, sc)
                            : cudaMemsetAsync(f->d_hstate, 0, zbytes, sc);
    if (e != cudaSuccess) return SOS_ECUDA;
    const long long nchunks = (n + chunk - 1) / chunk;
    for (long long i = 0; i < nchunks; ++i) {
        const int b = static_cast<int>(i % 3);
        const long long off = i * chunk;
        const long long len = (n - off) < chunk ? (n - off) : chunk;
        const size_t bytes = sizeof(float) * static_cast<size_t>(len);
        if (i >= 3 && cudaStreamWaitEvent(sin, f->ev_out[b], 0) != cudaSuccess) return SOS_ECUDA;
        if (cudaMemcpyAsync(f->hbuf[b], x_host + off, bytes, cudaMemcpyHostToDevice, sin) != cudaSuccess)
            return SOS_ECUDA;
        if (cudaEventRecord(f->ev_in[b], sin) != cudaSuccess) return SOS_ECUDA;
        if (cudaStreamWaitEvent(sc, f->ev_in[b], 0) != cudaSuccess) return SOS_ECUDA;
        const sos_status st = run_impl(f, f->hbuf[b], f->hbuf[b], len, f->d_hstate, f->d_hstate, sc);
        if (st != SOS_OK) return st;
        if (cudaEventRecord(f->ev_done[b], sc) != cudaSuccess) return SOS_ECUDA;
        if (cudaStreamWaitEvent(sout, f->ev_done[b], 0) != cudaSuccess) return SOS_ECUDA;
        if (cudaMemcpyAsync(y_host + off, f->hbuf[b], bytes, cudaMemcpyDeviceToHost, sout) != cudaSuccess)
            return SOS_ECUDA;
        if (cudaEventRecord(f->ev_out[b], sout) != cudaSuccess) return SOS_ECUDA;
    }
    if (zf_host) {
        if (cudaStreamSynchronize(sc) != cudaSuccess) return SOS_ECUDA;
        if (cudaMemcpy(zf_host, f->d_hstate, zbytes, cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
    }
    if (cudaStreamSynchronize(sout) != cudaSuccess || cudaStreamSynchronize(sc) != cudaSuccess) return SOS_ECUDA;
    f->last_stream = sc;
    return take_filter_status(f);  // reported once, as by sos_filter_sync_status
}

sos_status sos_filter_run_batch(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                float *const *y_dev, const int64_t *n, void *stream) {
    return run_batch_impl(n_signals, filters, x_dev, y_dev, n, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

sos_status sos_filter_run_batch_ex(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                   float *const *y_dev, const int64_t *n, const float *const *zi_dev,
                                   float *const *zf_dev, void *stream) {
    return run_batch_impl(n_signals, filters, x_dev, y_dev, n, zi_dev, zf_dev, static_cast<cudaStream_t>(stream));
}

sos_status sos_batch_plan_create(int n_signals, sos_filter *const *filters, const float *const *x_dev,
                                 float *const *y_dev, const int64_t *n, const float *const *zi_dev,
                                 float *const *zf_dev, sos_batch_plan **out) {
    return plan_create(n_signals, filters, x_dev, y_dev, n, zi_dev, zf_dev, out);
}

sos_status sos_batch_plan_launch(sos_batch_plan *p, void *stream) {
    if (!p) return SOS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(p->device) != cudaSuccess) return SOS_ECUDA;
    // fresh descriptors (tag 0 never matches) and tickets each launch: a launch enqueues no host work
    // and may be captured into a CUDA graph and replayed
    if (cudaMemsetAsync(p->d_desc, 0, sizeof(unsigned long long) * p->desc_words, s) != cudaSuccess ||
        cudaMemsetAsync(p->d_ticket, 0, sizeof(unsigned long long) * kBatchClasses, s) != cudaSuccess)
        return SOS_ECUDA;
    // one persistent launch over every class: the plan's queues, each class at offset 0 of its own
    // signal and tile arrays
    long long cls_sigs[kBatchClasses], cls_tiles[kBatchClasses], zero[kBatchClasses + 1] = {0};
    long long desc_off[kBatchClasses + 1] = {0};
    for (int c = 0; c < kBatchClasses; ++c) {
        cls_sigs[c] = p->tiles[c] ? 1 : 0;
        cls_tiles[c] = p->tiles[c];
        desc_off[c] = p->desc[c] ? p->desc[c] - p->d_desc : 0;
    }
    sosk::BatchAllParams ap;
    long long grid = 0;
    sos_status st = batch_all_params(cls_sigs, cls_tiles, zero, zero, desc_off, nullptr, nullptr, p->d_desc,
                                     p->d_ticket, 1u, p->d_status, p->device, ap, grid);
    if (st != SOS_OK) return st;
    for (int i = 0; i < ap.n_classes; ++i) {  // the plan keeps each class's arrays apart
        ap.q[i].sigs = p->sigs[ap.code[i]];
        ap.q[i].tile_sig = p->tile_sig[ap.code[i]];
    }
    if (sosk::launch_batch_all(ap, grid, s) != cudaSuccess) return SOS_ECUDA;
    return SOS_OK;
}

sos_status sos_batch_plan_status(sos_batch_plan *p) {
    if (!p) return SOS_EINVAL;
    if (cudaSetDevice(p->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SOS_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
    return (h & sosk::kDevErrTimeout) ? SOS_ETIMEOUT : SOS_OK;
}

sos_status sos_batch_plan_destroy(sos_batch_plan *p) {
    plan_free(p);
    return SOS_OK;
}

sos_status sos_batch_sync_status(int device) {
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SOS_ECUDA;
    return batch_status(device);
}

sos_status sos_autotune(int max_log2n, float *report) {
    if (max_log2n != 0 && (max_log2n < 16 || max_log2n > 28)) return SOS_EINVAL;
    const int top = max_log2n ? max_log2n : 28;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64) return SOS_ECUDA;
    const int64_t n_max = 1LL << top;
    float *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, sizeof(float) * n_max) != cudaSuccess || cudaMalloc(&y, sizeof(float) * n_max) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(x);
        return SOS_ENOMEM;
    }
    cudaMemset(x, 0, sizeof(float) * n_max);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        return SOS_ECUDA;
    }
    TuneTable tt;
    sos_status rc = SOS_OK;
    for (int K = 1; K <= sosk::kMaxPass && rc == SOS_OK; ++K) {
        // a stable cascade of K sections (the timing does not depend on the coefficients' values)
        std::vector<double> sos(5 * K);
        for (int k = 0; k < K; ++k) {
            const double r = 0.9 + 0.01 * k, th = 0.2 + 0.05 * k;
            const double c[5] = {0.05, 0.1, 0.05, -2.0 * r * std::cos(th), r * r};
            std::memcpy(&sos[5 * k], c, sizeof c);
        }
        for (int c = 0; c < kTuneCand && rc == SOS_OK; ++c) {
            sos_tuning t{};
            int solver = 0, N = 0, W = 0;
            candidate(c, &solver, &N, &W);
            t.solver = solver;
            t.N = N;
            t.groups_per_cta = solver == SOS_SOLVER_TC ? 0 : W;  // the tensor-core tile is fixed
            if (solver == SOS_SOLVER_CR) t.carry = SOS_CARRY_CASCADE;
            sos_filter *f = nullptr;
            rc = sos_filter_create(K, sos.data(), nullptr, &t, &f);
            if (rc != SOS_OK) break;
            for (int b = 0; b < kTuneBuckets && rc == SOS_OK; ++b) {
                if (kTuneLog2[b] > top) {
                    tt.gss[K - 1][b][c] = tt.gss[K - 1][b > 0 ? b - 1 : 0][c];
                    continue;
                }
                const int64_t n = 1LL << kTuneLog2[b];
                const int reps = n >= (1LL << 26) ? 3 : static_cast<int>((1LL << 26) / n);
                {
                    std::lock_guard<std::mutex> lk(f->mu);
                    for (int w = 0; w < 2 && rc == SOS_OK; ++w) rc = run_impl(f, x, y, n, nullptr, nullptr, st);
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < reps && rc == SOS_OK; ++r) rc = run_impl(f, x, y, n, nullptr, nullptr, st);
                    cudaEventRecord(e1, st);
                }
                float ms = 0.f;
                if (rc == SOS_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) !=
                                                                                     cudaSuccess))
                    rc = SOS_ECUDA;
                if (rc == SOS_OK) tt.gss[K - 1][b][c] = ms > 0.f ? static_cast<float>(n) * reps / ms / 1e6f : 0.f;
            }
            sos_filter_destroy(f);
        }
        for (int b = 0; b < kTuneBuckets; ++b) {
            int best = 0;
            for (int c = 1; c < kTuneCand; ++c)
                if (tt.gss[K - 1][b][c] > tt.gss[K - 1][b][best]) best = c;
            tt.best[K - 1][b] = static_cast<unsigned char>(best);
        }
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(x);
    cudaFree(y);
    if (rc != SOS_OK) return rc;
    tt.valid = true;
    if (report) std::memcpy(report, tt.gss, sizeof tt.gss);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[device] = tt;
    return SOS_OK;
}

sos_status sos_autotune_choice_ex(int n_sections, int64_t n, int *solver, int *N, int *groups_per_cta) {
    if (n_sections < 1 || !solver || !N) return SOS_EINVAL;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return SOS_ECUDA;
    int W = 0;
    if (!tuned_choice(device, n_sections, n, solver, N, &W)) {
        *solver = 0;
        *N = 0;
        W = 0;
    }
    if (groups_per_cta) *groups_per_cta = W;
    return SOS_OK;
}

sos_status sos_autotune_choice(int n_sections, int64_t n, int *solver, int *N) {
    return sos_autotune_choice_ex(n_sections, n, solver, N, nullptr);
}

sos_status sos_autotune_batch(float *report) {
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64) return SOS_ECUDA;
    constexpr int64_t kTotal = 1LL << 24;  // samples per timed batch
    float *x = nullptr, *y = nullptr;
    if (cudaMalloc(&x, sizeof(float) * kTotal) != cudaSuccess || cudaMalloc(&y, sizeof(float) * kTotal) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(x);
        return SOS_ENOMEM;
    }
    cudaMemset(x, 0, sizeof(float) * kTotal);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        return SOS_ECUDA;
    }
    BatchTune bt;
    sos_status rc = SOS_OK;
    for (int K = 1; K <= sosk::kMaxPass && rc == SOS_OK; ++K) {
        std::vector<double> sos(5 * K);  // a stable cascade (the timing does not depend on the values)
        for (int k = 0; k < K; ++k) {
            const double r = 0.9 + 0.01 * k, th = 0.2 + 0.05 * k;
            const double c[5] = {0.05, 0.1, 0.05, -2.0 * r * std::cos(th), r * r};
            std::memcpy(&sos[5 * k], c, sizeof c);
        }
        for (int g = 0; g < sosk::kBatchGeoms && rc == SOS_OK; ++g) {
            sos_tuning t{};
            t.N = sosk::batch_geom_n(g);  // pins the batch geometry of the filter's signals
            sos_filter *f = nullptr;
            rc = sos_filter_create(K, sos.data(), nullptr, &t, &f);
            if (rc != SOS_OK) break;
            for (int b = 0; b < kBatchTuneBuckets && rc == SOS_OK; ++b) {
                // equal signals filling kTotal samples, timed from a prepared plan (no host work
                // between the launches)
                const int64_t len = 1LL << kBatchTuneLog2[b];
                const int m = static_cast<int>(kTotal / len);
                std::vector<sos_filter *> fs(m, f);
                std::vector<const float *> xs(m);
                std::vector<float *> ys(m);
                std::vector<int64_t> ns(m, len);
                for (int i = 0; i < m; ++i) {
                    xs[i] = x + static_cast<int64_t>(i) * len;
                    ys[i] = y + static_cast<int64_t>(i) * len;
                }
                sos_batch_plan *plan = nullptr;
                rc = plan_create(m, fs.data(), xs.data(), ys.data(), ns.data(), nullptr, nullptr, &plan);
                if (rc != SOS_OK) break;
                constexpr int kReps = 5;
                for (int w = 0; w < 2 && rc == SOS_OK; ++w) rc = sos_batch_plan_launch(plan, st);
                cudaEventRecord(e0, st);
                for (int r = 0; r < kReps && rc == SOS_OK; ++r) rc = sos_batch_plan_launch(plan, st);
                cudaEventRecord(e1, st);
                float ms = 0.f;
                if (rc == SOS_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = SOS_ECUDA;
                if (rc == SOS_OK) rc = sos_batch_plan_status(plan);
                plan_free(plan);
                if (rc == SOS_OK) bt.gss[K - 1][b][g] = ms > 0.f ? static_cast<float>(kTotal) * kReps / ms / 1e6f : 0.f;
            }
            sos_filter_destroy(f);
        }
        for (int b = 0; b < kBatchTuneBuckets; ++b)
            bt.geom[K - 1][b] = bt.gss[K - 1][b][1] > bt.gss[K - 1][b][0] ? 1 : 0;
    }
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(x);
    cudaFree(y);
    if (rc != SOS_OK) return rc;
    bt.valid = true;
    if (report) std::memcpy(report, bt.gss, sizeof bt.gss);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_btune[device] = bt;
    return SOS_OK;
}

sos_status sos_autotune_batch_choice(int n_sections, int64_t n, int *N) {
    if (n_sections < 1 || !N) return SOS_EINVAL;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return SOS_ECUDA;
    const BatchGeomChoice gc = batch_geom_choice(device);
    *N = gc.valid ? sosk::batch_geom_n(gc.geom[(n_sections > sosk::kMaxPass ? sosk::kMaxPass : n_sections) - 1]
                                             [batch_tune_bucket(n)])
                  : 0;
    return SOS_OK;
}

sos_status sos_filter_stream_push(sos_filter *f, const float *x_dev, float *y_dev, int64_t n, void *stream) {
    if (!f) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    return run_impl(f, x_dev, y_dev, n, f->d_state, f->d_state, static_cast<cudaStream_t>(stream));
}

sos_status sos_filter_stream_state(sos_filter *f, float *z_out, const float *z_in, int on_device) {
    if (!f) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    if (cudaSetDevice(f->device) != cudaSuccess) return SOS_ECUDA;
    const size_t bytes = sizeof(float) * 2 * f->K;
    cudaStream_t s = f->last_stream;
    if (on_device) {
        if (z_out && cudaMemcpyAsync(z_out, f->d_state, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SOS_ECUDA;
        if (z_in && cudaMemcpyAsync(f->d_state, z_in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SOS_ECUDA;
    } else {
        if (cudaStreamSynchronize(s) != cudaSuccess) return SOS_ECUDA;
        if (z_out && cudaMemcpy(z_out, f->d_state, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
        if (z_in && cudaMemcpy(f->d_state, z_in, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return SOS_ECUDA;
    }
    int h = 0;
    if (!on_device) {
        if (cudaMemcpy(&h, f->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SOS_ECUDA;
        if (h & sosk::kDevErrTimeout) return SOS_ETIMEOUT;
    }
    return SOS_OK;
}

sos_status sos_filter_trace(sos_filter *f, uint64_t *buf_dev, int64_t capacity_blocks) {
    if (!f || capacity_blocks < 0) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    f->trace = reinterpret_cast<unsigned long long *>(buf_dev);
    f->trace_blocks = buf_dev ? capacity_blocks : 0;
    return SOS_OK;
}

sos_status sos_filter_sync_status(sos_filter *f) {
    if (!f) return SOS_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    if (cudaSetDevice(f->device) != cudaSuccess) return SOS_ECUDA;
    if (cudaStreamSynchronize(f->last_stream) != cudaSuccess) return SOS_ECUDA;
    return take_filter_status(f);
}

}  // extern "C"
