// Host side of the C ABI: geometry validation, FC parameters, frame layout,
// FP64 table generation (rounded once to FP32), job/chunk schedule, launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fc_internal.cuh"
#include "fc_trace.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return FC_ERR_CUDA;
}

constexpr size_t kSmemPerBlockMax = 232448;   // 227 KB opt-in dynamic + static limit on sm_10x
constexpr size_t kSmemPerSm = 233472;         // 228 KB shared memory per SM on sm_10x
constexpr size_t kSmemPerCtaReserve = 1024;   // shared memory the system keeps per resident CTA

// ---------------------------------------------------------------------------
// host staging of all device tables in one allocation
// ---------------------------------------------------------------------------
struct Blob {
  std::vector<unsigned char> bytes;
  size_t add(const void* p, size_t n, size_t align = 16) {
    size_t off = (bytes.size() + align - 1) / align * align;
    bytes.resize(off + n, 0);
    if (n && p) std::memcpy(bytes.data() + off, p, n);
    return off;
  }
  template <class T>
  size_t add_vec(const std::vector<T>& v) { return add(v.data(), v.size() * sizeof(T)); }
};

bool is_2a3b(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Radix schedule: all factors 3 as radix-3 passes (last); the power of two 2^a in
// ceil(a/4) balanced passes of at most radix 16. Fewer, larger passes beat smaller radices
// that would keep more of the CTA's threads busy, because each pass costs two CTA
// barriers: schedules with at least 256 butterflies per pass (radix 4 for one 1024-point
// transform) made the 20 MHz symbol-sync TX kernel 33 % slower.
void radix_plan(int n, unsigned char* radix, int* npass) {
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  int k = 0;
  if (a > 0) {
    const int passes = (a + 3) / 4;
    const int base = a / passes, extra = a % passes;
    for (int i = 0; i < passes; ++i) radix[k++] = (unsigned char)(1 << (base + (i < extra ? 1 : 0)));
  }
  for (int i = 0; i < b; ++i) radix[k++] = 3;
  *npass = k;
}

// Candidate radix schedules of an n-point transform for the autotuner: the power of two
// 2^a split into ceil(a/4) or ceil(a/4) + 1 passes of radix 2..16, balanced with the
// larger radices first or last, or as many radix-16 passes as fit first; the radix-3
// passes last (as radix_plan) or first. The rule's own schedule comes first.
std::vector<std::vector<unsigned char>> radix_candidates(int n) {
  std::vector<std::vector<unsigned char>> out;
  auto add = [&](const std::vector<unsigned char>& r) {
    if ((int)r.size() > FC_MAX_PASSES) return;
    if (std::find(out.begin(), out.end(), r) == out.end()) out.push_back(r);
  };
  {
    unsigned char r[FC_MAX_PASSES];
    int np = 0;
    radix_plan(n, r, &np);
    add(std::vector<unsigned char>(r, r + np));
  }
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  std::vector<std::vector<unsigned char>> twos;
  if (a == 0) twos.push_back({});
  for (int passes = (a + 3) / 4; a > 0 && passes <= (a + 3) / 4 + 1 && passes <= a; ++passes) {
    const int base = a / passes, extra = a % passes;
    std::vector<unsigned char> big_first, big_last;
    for (int i = 0; i < passes; ++i) big_first.push_back((unsigned char)(1 << (base + (i < extra ? 1 : 0))));
    big_last.assign(big_first.rbegin(), big_first.rend());
    twos.push_back(big_first);
    twos.push_back(big_last);
  }
  if (a > 4) {                                         // radix 16 while it fits, then the rest
    std::vector<unsigned char> r;
    int left = a;
    while (left >= 4) { r.push_back(16); left -= 4; }
    if (left) r.push_back((unsigned char)(1 << left));
    twos.push_back(r);
  }
  for (const auto& t : twos) {
    std::vector<unsigned char> last = t, first(b, 3);
    for (int i = 0; i < b; ++i) last.push_back(3);
    first.insert(first.end(), t.begin(), t.end());
    add(last);
    add(first);
  }
  return out;
}

struct SubHost {
  int L = 0, Lo = 0, Lact = 0, c = 0, g = 0;
  int L_O = 0, L_S = 0, L_L = 0, L_T = 0, S_L = 0, n_low = 0, R = 0;
  std::vector<double> D;
  std::vector<int> lcp, soff;
};

struct GroupHost {
  int N = 0, N_O = 0, N_S = 0, N_L = 0, N_T = 0, B = 0, lead_hi = 0, T_lead = 0, len = 0, R = 0, offset = 0;
  std::vector<int> ncp, sigma, cps;
  std::vector<int> subs;
};

}  // namespace

// Launch shape of one call: split index (chunks per stream), the generic kernels instead
// of the specialised or tensor-core ones, and the generic-kernel set (-1: by the call's CTA
// count, see gen_for)
struct Choice {
  int split = 0;
  int generic = 0;
  int set = -1;
};

struct fc_plan {
  int device = 0;
  int num_sms = 0;
  size_t smem_cap = kSmemPerBlockMax - sizeof(FcPlanDev) - 256;   // dynamic shared memory per CTA
  size_t smem_sm = kSmemPerSm;              // shared memory per SM
  // generic-kernel sets (0: 512-thread CTAs, one per SM; 1: 256, two per SM; 2: 128, four
  // per SM) and which of them the plan's transforms and shared memory fit (0 always)
  const FcGenKernels* gen[3] = {nullptr, nullptr, nullptr};
  bool gen_fits[3] = {true, false, false};
  FcPlanDev h{};
  FcPlanDev* d_plan = nullptr;
  unsigned char* d_mem = nullptr;
  FcJob* d_jobs = nullptr;
  int n_jobs = 0;
  std::vector<int> splits;                  // chunk counts per stream available
  std::vector<const FcChunk*> tx_chunks, rx_chunks;
  std::vector<int> tx_nchunks, rx_nchunks;
  int io = 0;                               // FC_IO_* bits of the frame calls (FC_FLAG_IO_BF16)
  bool warp_path = false;                   // warp-specialised symbol-sync kernels apply
  bool cont_warp_tx = false, cont_warp_rx = false;   // warp-specialised continuous kernels apply (per direction)
  bool tc_tx = false, tc_rx = false;        // tensor-core FC passes apply (FC_FLAG_TENSOR_DFT)
  bool tc_ofdm = false;                     // and the OFDM (I)DFT too (L_OFDM = 4096)
  const unsigned char* d_dft64 = nullptr;   // DFT-64 B operand images (hi, lo)
  int* d_err = nullptr;                     // device error word of the tensor-core kernels
  unsigned tc_first_wait = 1u << 22;        // poll limit of the tensor-core kernels' first GEMM wait
  FcJob* d_wjobs = nullptr;                 // one stream's TX jobs in dealing order (warp kernels, BF16 input)
  int n_wjobs_big = 0;                      // the first n_wjobs_big of them belong to N = 2048 groups
  int n_wjobs_init = 0;                     // of which the first n_wjobs_init initialise the TX waveform
  FcJob* d_wpjobs = nullptr;                // the same list with the N = 1024 symbols in pairs
  int n_wpjobs = 0;
  FcJob* d_wrxjobs = nullptr;               // the RX list: by time, N = 1024 symbols in pairs
  int n_wrxjobs = 0;
  int warp_weight_floats = 0;               // sum over groups of the subband length (warp TX weights)
  size_t smem_tx = 0, smem_rx = 0, smem_ofdm = 0;
  int syms_per_stream = 0;
  fc_sizes sizes{};
  // launch choices measured by fc_plan_autotune, per (n_streams, direction); execute
  // calls without an entry use the occupancy heuristic pick_split
  mutable std::mutex tune_mu;
  std::map<std::pair<int, int>, Choice> tuned;
};

namespace {

int build_plan(fc_plan* pl, const fc_geometry* geo, bool upload) {
  if (!geo) return fail(FC_ERR_INVALID, "geometry is NULL");
  if (geo->mode != FC_CONTINUOUS && geo->mode != FC_SYMBOL_SYNC) return fail(FC_ERR_INVALID, "unknown mode");
  if ((geo->scheme_tx != FC_OLA && geo->scheme_tx != FC_OLS) || (geo->scheme_rx != FC_OLA && geo->scheme_rx != FC_OLS))
    return fail(FC_ERR_INVALID, "unknown OLA/OLS scheme");
  if (geo->n_groups < 1 || geo->n_groups > FC_MAX_GROUPS || !geo->groups)
    return fail(FC_ERR_INVALID, "n_groups out of range");
  if (geo->n_subbands < 1 || geo->n_subbands > FC_MAX_SUBBANDS || !geo->subbands)
    return fail(FC_ERR_INVALID, "n_subbands out of range");
  const bool sync = geo->mode == FC_SYMBOL_SYNC;
  const int G = geo->n_groups, M = geo->n_subbands;

  // ---- groups --------------------------------------------------------------
  std::vector<GroupHost> gh(G);
  for (int g = 0; g < G; ++g) {
    const fc_group& in = geo->groups[g];
    GroupHost& o = gh[g];
    o.N = in.n_long;
    o.N_O = in.n_overlap;
    o.B = in.n_symbols;
    if (o.N < 2 || o.N_O < 0 || o.N_O >= o.N) return fail(FC_ERR_INVALID, "need 0 <= N_O < N");
    if (o.B < 1 || !in.n_cp) return fail(FC_ERR_INVALID, "need n_symbols >= 1 and n_cp");
    if (!is_2a3b(o.N) || o.N > FC_MAX_TRANSFORM) return fail(FC_ERR_UNSUPPORTED, "N must be 2^a 3^b <= 4096");
    o.N_S = o.N - o.N_O;
    o.N_L = (o.N_O + 1) / 2;   // ceil(N_O/2)
    o.N_T = o.N_O / 2;
    o.ncp.assign(in.n_cp, in.n_cp + o.B);
    for (int v : o.ncp)
      if (v < 0) return fail(FC_ERR_INVALID, "negative N_CP");
    if (sync) {
      if (2 * o.N_O != o.N || o.N % 4) return fail(FC_ERR_INVALID, "symbol-sync needs N_O = N/2 and 4 | N");
      for (int v : o.ncp)
        if (v > o.N / 4) return fail(FC_ERR_INVALID, "symbol-sync needs N_CP,n <= N/4");
    }
    o.lead_hi = (in.lead_pad < 0) ? o.N_O : in.lead_pad;
  }

  // ---- subbands ------------------------------------------------------------
  std::vector<SubHost> sh(M);
  for (int m = 0; m < M; ++m) {
    const fc_subband& in = geo->subbands[m];
    SubHost& o = sh[m];
    o.L = in.l_short; o.Lo = in.l_ofdm; o.Lact = in.n_active; o.c = in.centre_bin; o.g = in.group;
    if (o.g < 0 || o.g >= G) return fail(FC_ERR_INVALID, "subband group out of range");
    const GroupHost& g = gh[o.g];
    if (!in.weights) return fail(FC_ERR_INVALID, "weights is NULL");
    if (o.L < 1 || o.L > g.N) return fail(FC_ERR_INVALID, "need 1 <= L <= N");
    if (!is_2a3b(o.L) || !is_2a3b(o.Lo) || o.Lo > FC_MAX_TRANSFORM)
      return fail(FC_ERR_UNSUPPORTED, "L and L_OFDM must be 2^a 3^b <= 4096");
    if (o.Lact < 1 || o.Lact > o.Lo) return fail(FC_ERR_INVALID, "need 1 <= L_act <= L_OFDM");
    if ((long long)g.N_O * o.L % g.N) return fail(FC_ERR_INVALID, "L_O = N_O L / N is not an integer");
    o.L_O = (int)((long long)g.N_O * o.L / g.N);
    o.L_S = o.L - o.L_O;
    o.L_L = (o.L_O + 1) / 2;
    o.L_T = o.L_O / 2;
    o.D.assign(in.weights, in.weights + o.L);
    o.lcp.resize(g.B);
    for (int n = 0; n < g.B; ++n) {
      const long long num = (long long)g.ncp[n] * o.L;
      if (!sync && num % g.N) return fail(FC_ERR_INVALID, "continuous FC needs integer low-rate CPs (N_CP L / N)");
      o.lcp[n] = (int)(num / g.N);   // floor, Sec. III-E
    }
    if (sync) {
      if (o.L % 4) return fail(FC_ERR_INVALID, "symbol-sync needs 4 | L");
      if (o.Lo != o.L) return fail(FC_ERR_INVALID, "symbol-sync needs L_OFDM = L");
      o.soff.resize(g.B);                 // symbol starts of the time-domain I/O
      int acc = 0;
      for (int n = 0; n < g.B; ++n) {
        o.soff[n] = acc;
        acc += o.lcp[n] + o.Lo;
      }
    } else {
      if ((long long)o.Lo * g.N % o.L) return fail(FC_ERR_INVALID, "N_OFDM = L_OFDM N / L is not an integer");
      if ((long long)g.lead_hi * o.L % g.N) return fail(FC_ERR_INVALID, "lead pad is not an integer at low rate");
      o.S_L = (int)((long long)g.lead_hi * o.L / g.N);
      if (o.S_L < o.L_L) return fail(FC_ERR_INVALID, "lead pad shorter than L_L");
      o.soff.resize(g.B);
      int acc = 0;
      for (int n = 0; n < g.B; ++n) {
        o.soff[n] = acc;
        acc += o.lcp[n] + o.Lo;
      }
      o.n_low = acc;
      const long long u0 = (long long)o.n_low + 2LL * o.S_L;
      o.R = (u0 <= o.L) ? 1 : (int)((u0 - o.L + o.L_S - 1) / o.L_S) + 1;
    }
  }
  for (int g = 0; g < G; ++g) {
    for (int m = 0; m < M; ++m)
      if (sh[m].g == g) gh[g].subs.push_back(m);
    if (gh[g].subs.empty()) return fail(FC_ERR_INVALID, "a group has no subband");
  }
  // subbands must be stored grouped for the kernels; keep the caller's grid
  // order through grid_off, and sort the processing order by group
  std::vector<int> order;
  for (int g = 0; g < G; ++g)
    for (int m : gh[g].subs) order.push_back(m);

  // ---- frame layout --------------------------------------------------------
  for (int g = 0; g < G; ++g) {
    GroupHost& o = gh[g];
    if (sync) {
      o.T_lead = o.N / 4 - o.ncp[0];
      long long q = (long long)o.N / 2 + (long long)o.B * o.N;
      for (int n = 1; n < o.B; ++n) q += o.ncp[n];
      o.len = (int)q;                                         // eq:waveformLen
      o.sigma.resize(o.B);
      long long acc = 0;
      for (int n = 0; n < o.B; ++n) {
        if (n > 0) acc += o.ncp[n];
        o.sigma[n] = (int)((long long)n * o.N + acc);        // eq:multi-symb
      }
    } else {
      const SubHost& s0 = sh[o.subs[0]];
      for (int m : o.subs) {
        const long long dur_hi = (long long)sh[m].n_low * o.N / sh[m].L;
        const long long dur0 = (long long)s0.n_low * o.N / s0.L;
        if (dur_hi != dur0 || sh[m].R != s0.R)
          return fail(FC_ERR_INVALID, "continuous subbands of one group need equal high-rate durations");
      }
      o.R = s0.R;
      o.T_lead = o.lead_hi;
      o.len = (o.R - 1) * o.N_S + o.N;
    }
    o.cps.resize(o.B);
    long long acc = 0;
    for (int n = 0; n < o.B; ++n) {
      if (n > 0) acc += o.ncp[n];
      o.cps[n] = (int)(acc % o.N);
    }
  }
  int t_s = 0;
  for (auto& o : gh) t_s = std::max(t_s, o.T_lead);
  long long frame_len = 0;
  for (auto& o : gh) {
    o.offset = t_s - o.T_lead;
    frame_len = std::max(frame_len, (long long)o.offset + o.len);
  }
  if (frame_len > (1LL << 30)) return fail(FC_ERR_UNSUPPORTED, "frame too long");

  // ---- stream calls (fc_state): a slot is the whole CP list of every group ----
  // The K-slot frame is the one-slot frame repeated at period T (so a stream call can
  // run the one-slot frame and carry D = Q - T samples) when every group lasts the
  // same T, c_m T / N is an integer (theta_n and phi_r repeat every slot) and, in
  // continuous mode, a slot is a whole number of hops L_S with S_L >= L_O (the one-
  // slot frame then holds every block that touches its symbols).
  long long slot_len = -1;
  bool streamable = true;
  for (int m = 0; m < M; ++m) {
    const GroupHost& g = gh[sh[m].g];
    long long t = 0;
    for (int n = 0; n < g.B; ++n) t += g.ncp[n];
    t += sync ? (long long)g.B * g.N : (long long)g.B * sh[m].Lo * g.N / sh[m].L;
    if (slot_len < 0) slot_len = t;
    if (t != slot_len || ((long long)sh[m].c * t) % g.N) streamable = false;
    if (!sync && (sh[m].n_low % sh[m].L_S || sh[m].S_L < sh[m].L_O)) streamable = false;
  }
  const long long stream_delay = frame_len - slot_len;
  if (stream_delay < 0 || stream_delay > slot_len) streamable = false;

  // ---- transform sizes, twiddles ------------------------------------------
  std::vector<int> sizes;
  auto size_index = [&](int n) {
    for (size_t i = 0; i < sizes.size(); ++i)
      if (sizes[i] == n) return (int)i;
    sizes.push_back(n);
    return (int)sizes.size() - 1;
  };
  std::vector<int> g_sizeN(G), s_sizeL(M), s_sizeO(M);
  for (int g = 0; g < G; ++g) g_sizeN[g] = size_index(gh[g].N);
  for (int m = 0; m < M; ++m) {
    s_sizeL[m] = size_index(sh[m].L);
    s_sizeO[m] = size_index(sh[m].Lo);
  }
  if ((int)sizes.size() > FC_MAX_SIZES) return fail(FC_ERR_UNSUPPORTED, "too many distinct transform sizes");

  Blob blob;
  std::vector<size_t> tw_off(sizes.size());
  for (size_t i = 0; i < sizes.size(); ++i) {
    const int n = sizes[i];
    std::vector<float2> tw(n);
    for (int mm = 0; mm < n; ++mm) {
      const double ang = 2.0 * M_PI * (double)mm / (double)n;   // exact reduction: mm < n
      tw[mm] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    tw_off[i] = blob.add_vec(tw);
  }

  // ---- per-subband tables --------------------------------------------------
  std::vector<size_t> off_dtx(M), off_drx(M), off_lcp(M), off_soff(M);
  std::vector<int> plo(M), phi(M);
  for (int m = 0; m < M; ++m) {
    const SubHost& o = sh[m];
    const GroupHost& g = gh[o.g];
    const double I = (double)g.N / (double)o.L;
    const double stx = std::sqrt(I) / (std::sqrt((double)o.Lo) * (double)g.N);
    const double srx = 1.0 / (std::sqrt(I) * (double)o.L * std::sqrt((double)o.Lo));
    std::vector<float> dtx(o.L), drx(o.L);
    int lo = o.L, hi = 0;
    for (int p = 0; p < o.L; ++p) {
      dtx[p] = (float)(o.D[p] * stx);
      drx[p] = (float)(o.D[p] * srx);
      if (o.D[p] != 0.0) {
        lo = std::min(lo, p);
        hi = std::max(hi, p + 1);
      }
    }
    if (lo >= hi) lo = hi = 0;
    plo[m] = lo;
    phi[m] = hi;
    off_dtx[m] = blob.add_vec(dtx);
    off_drx[m] = blob.add_vec(drx);
    off_lcp[m] = blob.add_vec(o.lcp);
    std::vector<int> so = o.soff;
    if (so.empty()) so.assign(1, 0);
    off_soff[m] = blob.add_vec(so);
  }
  std::vector<size_t> off_sigma(G), off_ncp(G), off_cps(G);
  for (int g = 0; g < G; ++g) {
    std::vector<int> sg = gh[g].sigma;
    if (sg.empty()) sg.assign(1, 0);
    off_sigma[g] = blob.add_vec(sg);
    off_ncp[g] = blob.add_vec(gh[g].ncp);
    off_cps[g] = blob.add_vec(gh[g].cps);
  }

  // ---- jobs ----------------------------------------------------------------
  std::vector<FcJob> jobs;
  std::vector<int> span;
  for (int g = 0; g < G; ++g) {
    const GroupHost& o = gh[g];
    if (sync) {
      for (int n = 0; n < o.B; ++n) jobs.push_back(FcJob{g, n, 2, o.offset + o.sigma[n]});
    } else {
      for (int r0 = 0; r0 < o.R; r0 += 2) jobs.push_back(FcJob{g, r0, std::min(2, o.R - r0), o.offset + r0 * o.N_S});
    }
  }
  std::stable_sort(jobs.begin(), jobs.end(), [](const FcJob& a, const FcJob& b) { return a.start < b.start; });
  int max_span = 0;
  for (const FcJob& jb : jobs) {
    const GroupHost& o = gh[jb.group];
    const int sp = sync ? 3 * o.N / 2 : (jb.nblk - 1) * o.N_S + o.N;
    span.push_back(sp);
    max_span = std::max(max_span, sp);
  }
  const int n_jobs = (int)jobs.size();
  const size_t off_jobs = blob.add_vec(jobs);

  // chunk tables for several splits per stream
  std::vector<int> splits;
  for (int k = 1; k <= 64 && k <= n_jobs; k *= 2) splits.push_back(k);
  std::vector<size_t> off_txc, off_rxc;
  std::vector<int> ntx, nrx;
  for (int K : splits) {
    std::vector<int> bidx;   // job index boundaries
    for (int c = 0; c <= K; ++c) bidx.push_back((int)((long long)c * n_jobs / K));
    // TX: owned time ranges start at the first job of each chunk
    std::vector<int> tb;
    tb.push_back(0);
    for (int c = 1; c < K; ++c) {
      const int t = jobs[bidx[c]].start;
      if (t > tb.back()) tb.push_back(t);
    }
    tb.push_back((int)frame_len);
    std::vector<FcChunk> tx;
    for (size_t c = 0; c + 1 < tb.size(); ++c) {
      const int t0 = tb[c], t1 = tb[c + 1];
      int j0 = 0;
      while (j0 < n_jobs && (long long)jobs[j0].start + max_span <= t0) ++j0;
      int j1 = j0;
      while (j1 < n_jobs && jobs[j1].start < t1) ++j1;
      tx.push_back(FcChunk{j0, j1, t0, t1});
    }
    std::vector<FcChunk> rx;
    for (int c = 0; c < K; ++c)
      if (bidx[c + 1] > bidx[c]) rx.push_back(FcChunk{bidx[c], bidx[c + 1], 0, 0});
    off_txc.push_back(blob.add_vec(tx));
    off_rxc.push_back(blob.add_vec(rx));
    ntx.push_back((int)tx.size());
    nrx.push_back((int)rx.size());
  }

  // warp-specialised path: symbol-sync, one subband per group, I = 2, L in {512, 1024}
  // (complex-BF16 I/O: the TX kernel accumulates into a complex64 waveform in the
  // workspace, rounded once into the BF16 output afterwards)
  const bool io_time = (geo->flags & FC_FLAG_IO_TIME) != 0;
  const bool io_bf16 = (geo->flags & FC_FLAG_IO_BF16) != 0;
  bool warp_ok = sync && !(geo->flags & FC_FLAG_GENERIC_KERNELS) && !io_time && (frame_len % 2 == 0);
  for (int g = 0; g < G && warp_ok; ++g) {
    if (gh[g].subs.size() != 1) { warp_ok = false; break; }
    const SubHost& o = sh[gh[g].subs[0]];
    const bool shape = (o.L == 1024 && gh[g].N == 2048) || (o.L == 512 && gh[g].N == 1024);
    if (!shape) warp_ok = false;
  }
  // warp-specialised continuous path: one group, one subband, L = L_OFDM = 384, N = 512,
  // 50 % overlap, the group at the frame's start; per direction when that side is
  // overlap-save (its outputs are disjoint and written once)
  bool cont_warp = !sync && G == 1 && M == 1 && !io_time && !(geo->flags & FC_FLAG_GENERIC_KERNELS) &&
                   sh[0].L == 384 && sh[0].Lo == 384 && gh[0].N == 512 && 2 * gh[0].N_O == gh[0].N &&
                   gh[0].offset == 0;
  size_t off_wjobs = 0, off_wtx = 0, off_wrx = 0;
  int n_big = 0, n_wtx = 0, n_init = 0, n_wrx = 0;
  if (warp_ok) {
    // One stream's jobs in the order the warp kernels deal them (the job-major list of
    // all streams), most expensive first: the N = 2048 groups' symbols, then the N = 1024
    // groups'. RX takes them by time, the N = 1024 symbols in pairs (n, n + 1) (nblk = 4)
    // whose OFDM DFTs share one two-transform FFT (a group's odd last symbol alone). TX
    // takes the same pairs (their OFDM IDFTs; with complex64 input, else single symbols)
    // and, with one N = 2048 group, that group's even symbols first: their launch
    // initialises the waveform (stores, and zeros between their disjoint spans) instead
    // of a memset.
    int big_groups = 0;
    for (const GroupHost& o : gh) big_groups += o.N == 2048;
    std::vector<FcJob> big, init, rest, singles, pairs;
    for (const FcJob& jb : jobs) {                   // jobs are sorted by time
      if (gh[jb.group].N != 2048) {
        singles.push_back(jb);
        continue;
      }
      big.push_back(jb);
      (big_groups == 1 && jb.index % 2 == 0 ? init : rest).push_back(jb);
    }
    for (int g = 0; g < G; ++g) {
      const GroupHost& o = gh[g];
      if (o.N == 2048) continue;
      for (int n = 0; n < o.B; n += 2) pairs.push_back(FcJob{g, n, n + 1 < o.B ? 4 : 2, o.offset + o.sigma[n]});
    }
    std::stable_sort(pairs.begin(), pairs.end(), [](const FcJob& a, const FcJob& b) { return a.start < b.start; });
    n_big = (int)big.size();
    n_init = (int)init.size();
    auto cat = [](std::vector<FcJob> a, const std::vector<FcJob>& b, const std::vector<FcJob>& c) {
      a.insert(a.end(), b.begin(), b.end());
      a.insert(a.end(), c.begin(), c.end());
      return a;
    };
    const std::vector<FcJob> tx_singles = cat(init, rest, singles), tx_pairs = cat(init, rest, pairs);
    const std::vector<FcJob> rx = cat(big, {}, pairs);
    off_wjobs = blob.add_vec(tx_singles);
    off_wtx = blob.add_vec(tx_pairs);
    off_wrx = blob.add_vec(rx);
    n_wtx = (int)tx_pairs.size();
    n_wrx = (int)rx.size();
  }

  // ---- buffers and shared memory -------------------------------------------
  int n_max = 0, l_max = 0, lo_max = 0;
  for (auto& o : gh) n_max = std::max(n_max, o.N);
  for (auto& o : sh) {
    l_max = std::max(l_max, o.L);
    lo_max = std::max(lo_max, o.Lo);
  }
  // in-place FFT capacity of a CTA of `threads` threads: batch 2 of N and L
  auto fits_fft = [&](int threads) {
    for (int n : sizes) {
      const int cap = (n % 3 == 0) ? threads * (FC_MAX_ELEMS_PER_THREAD / 3) * 3 : threads * FC_MAX_ELEMS_PER_THREAD;
      if (2 * n > cap) return false;
    }
    return true;
  };
  if (!fits_fft(512)) return fail(FC_ERR_UNSUPPORTED, "transform too large for the in-place FFT");
  // TX ring: the longest job span (at least one sample per thread), a multiple of 16;
  // transform buffers padded (fc_padded_len): symbol-sync W holds L then 2L (TX: OFDM
  // symbol and the two segments; RX: the two short blocks and the concatenated body),
  // continuous W the 2L of a block pair
  auto ring_for = [&](int threads) { return (std::max(max_span, threads) + 15) / 16 * 16; };
  const int ybuf = fc_padded_len(2 * n_max);
  const int wbuf = sync ? fc_padded_len(l_max) + fc_padded_len(2 * l_max) : fc_padded_len(2 * l_max);
  // generic kernels: which CTA sizes (128 threads four per SM, 256 two per SM, 512 one per
  // SM) hold every transform in their in-place FFT and fit their shared memory as many
  // times per SM; several CTAs per SM overlap one CTA's barrier waits with the others'
  // work, larger CTAs finish one chunk sooner (the choice per call is gen_for's)
  const size_t static_smem = sizeof(FcPlanDev) + 256;
  const int ring = ring_for(512);            // serves every set (ring >= the CTA's threads)
  auto fits_sm = [&](int threads, int per_sm) {
    const size_t budget = pl->smem_sm / per_sm;
    const size_t need = (size_t)(ring + ybuf + wbuf) * sizeof(float2) + static_smem + kSmemPerCtaReserve;
    return fits_fft(threads) && need <= budget;
  };
  pl->gen[0] = &fc_gen_kernels_512();
  pl->gen[1] = &fc_gen_kernels_256();
  pl->gen[2] = &fc_gen_kernels_128();
  pl->gen_fits[1] = fits_sm(256, 2);
  pl->gen_fits[2] = fits_sm(128, 4);
  pl->smem_tx = (size_t)(ring + ybuf + wbuf) * sizeof(float2);
  pl->smem_rx = (size_t)(ybuf + wbuf) * sizeof(float2);
  pl->smem_ofdm = (size_t)fc_padded_len(lo_max) * sizeof(float2);
  const size_t smem_cap = pl->smem_cap;
  if (pl->smem_tx > smem_cap || pl->smem_rx > smem_cap)
    return fail(FC_ERR_UNSUPPORTED, "geometry needs more shared memory than one SM has");

  // tensor-core FC passes: continuous, one group, one subband, L = N = 4096; RX only
  // for overlap-save (the OLA analysis keeps the FP32 kernels)
  const bool tc_tx = (geo->flags & FC_FLAG_TENSOR_DFT) && !io_bf16 && !sync && G == 1 && M == 1 && sh[0].L == 4096 &&
                     gh[0].N == 4096;
  const bool tc_rx = tc_tx && geo->scheme_rx == FC_OLS;

  // workspace (continuous): low-rate stream per subband, or R*L per subband for RX OLA;
  // the tensor-core passes add R rows of 4096 bins between their two transforms
  long long ws_len = 0;
  std::vector<long long> ws_off(M, 0);
  if (!sync) {
    for (int m : order) {
      ws_off[m] = ws_len;
      long long need = sh[m].n_low;
      if (geo->scheme_rx == FC_OLA) need = std::max(need, (long long)sh[m].R * sh[m].L);
      ws_len += (need + 1) / 2 * 2;   // keep 16-byte alignment per slot
    }
  }
  long long tc_off = 0;
  if (tc_tx) {
    tc_off = ws_len;
    ws_len += (long long)sh[0].R * 4096;
  }
  // the warp kernels' complex64 frame: the TX accumulator of a BF16 output, the RX copy
  // of a BF16 input
  if (warp_ok && io_bf16) ws_len = std::max(ws_len, ((long long)frame_len + 1) / 2 * 2);

  // grid offsets in the caller's subband order
  std::vector<long long> grid_off(M);
  long long grid_len = 0;
  for (int m = 0; m < M; ++m) {
    grid_off[m] = grid_len;
    grid_len += (long long)gh[sh[m].g].B * sh[m].Lact;
  }

  int syms = 0;
  for (int m = 0; m < M; ++m) syms += gh[sh[m].g].B;
  pl->syms_per_stream = syms;

  fc_sizes& z = pl->sizes;
  z.grid_len = grid_len;
  z.wave_len = frame_len;
  {
    const GroupHost& o = gh[0];
    const SubHost& s0 = sh[o.subs[0]];
    long long nom = 0;
    const long long n_ofdm = sync ? o.N : (long long)s0.Lo * o.N / s0.L;
    for (int n = 0; n < o.B; ++n) nom += n_ofdm + o.ncp[n];
    z.nominal_len = nom;
  }
  z.workspace_per_stream = ws_len * (long long)sizeof(float2);
  // time-domain I/O layout: per subband (creation order) every symbol's CP and body (TX)
  // or body (RX)
  std::vector<long long> t_tx_off(M), t_rx_off(M);
  long long t_tx = 0, t_rx = 0;
  for (int m = 0; m < M; ++m) {
    const GroupHost& g = gh[sh[m].g];
    t_tx_off[m] = t_tx;
    t_rx_off[m] = t_rx;
    for (int n = 0; n < g.B; ++n) t_tx += sh[m].lcp[n] + sh[m].Lo;
    t_rx += (long long)g.B * sh[m].Lo;
  }
  if (t_tx > 0x7fffffffLL || t_rx > 0x7fffffffLL) return fail(FC_ERR_UNSUPPORTED, "time-domain I/O too long");
  z.time_tx_len = t_tx;
  z.time_rx_len = t_rx;
  z.tx_in_len = io_time ? t_tx : grid_len;
  z.rx_out_len = io_time ? t_rx : grid_len;
  z.sample_bytes = io_bf16 ? 4 : 8;
  pl->io = io_bf16 ? (FC_IO_IN_BF16 | FC_IO_OUT_BF16) : 0;
  z.slot_len = streamable ? slot_len : 0;
  z.stream_delay = streamable ? stream_delay : 0;
  // the one-warp kernels: one launch per job shape present (TX: the N = 2048 jobs in two
  // launches where the first initialises the waveform), + the BF16 rounding / widening pass
  int warp_shapes = 0;
  if (warp_ok) {
    bool big = false, small = false;
    for (const GroupHost& o : gh) (o.N == 2048 ? big : small) = true;
    warp_shapes = (int)big + (int)small;
  }
  z.tx_kernels = sync ? (warp_ok ? warp_shapes + (n_init > 0 && n_init < n_big) + (int)io_bf16 : 1) : (tc_tx ? 3 : 2);
  z.rx_kernels = sync ? (warp_ok ? warp_shapes + (int)io_bf16 : 1) : (tc_rx ? 3 : 2);
  size_t off_dft = 0, off_err = 0;
  if (tc_tx) {
    std::vector<unsigned char> img(fc_tc_dft64_image_bytes());
    fc_tc_dft64_image(img.data());
    off_dft = blob.add(img.data(), img.size(), 256);
    const int zero = 0;
    off_err = blob.add(&zero, sizeof(int));
  }
  // ---- device upload ---------------------------------------------------------
  const size_t off_plan = blob.add(nullptr, sizeof(FcPlanDev));
  // Without upload (host-only check) every table pointer is laid out against a
  // null base, so the whole host path runs and only the two CUDA calls are skipped.
  if (upload) {
    cudaError_t e = cudaMalloc(&pl->d_mem, blob.bytes.size());
    if (e != cudaSuccess) {
      pl->d_mem = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(FC_ERR_NOMEM, "cudaMalloc of plan tables failed")
                                            : cuda_fail(e, "cudaMalloc");
    }
  }
  unsigned char* base = pl->d_mem;
  FcPlanDev& P = pl->h;
  std::memset(&P, 0, sizeof(P));
  P.mode = geo->mode;
  P.scheme_tx = geo->scheme_tx;
  P.scheme_rx = geo->scheme_rx;
  P.flags = geo->flags;
  P.n_groups = G;
  P.n_subs = M;
  P.n_sizes = (int)sizes.size();
  P.frame_len = (int)frame_len;
  P.grid_len = grid_len;
  P.ws_len = ws_len;
  P.tc_off = tc_off;
  P.time_tx_len = (int)t_tx;
  P.time_rx_len = (int)t_rx;
  P.ring = ring;
  P.ybuf = ybuf;
  P.wbuf = wbuf;
  P.max_span = max_span;
  for (size_t i = 0; i < sizes.size(); ++i) {
    FcSize& z = P.sz[i];
    z.n = sizes[i];
    radix_plan(z.n, z.radix, &z.npass);
    z.tw = reinterpret_cast<const float2*>(base + tw_off[i]);
  }
  // kernels walk subbands of a group contiguously: store them in group order
  std::vector<int> slot_of(M);
  for (int i = 0; i < M; ++i) slot_of[order[i]] = i;
  int first = 0;
  for (int g = 0; g < G; ++g) {
    const GroupHost& o = gh[g];
    FcGroupDev& d = P.g[g];
    d.N = o.N; d.N_O = o.N_O; d.N_S = o.N_S; d.N_L = o.N_L; d.N_T = o.N_T;
    d.B = o.B; d.offset = o.offset; d.len = o.len; d.R = o.R;
    d.size_N = g_sizeN[g];
    d.first_sub = first;
    d.n_sub = (int)o.subs.size();
    first += d.n_sub;
    d.sigma = reinterpret_cast<const int*>(base + off_sigma[g]);
    d.ncp = reinterpret_cast<const int*>(base + off_ncp[g]);
    d.cps = reinterpret_cast<const int*>(base + off_cps[g]);
  }
  for (int m = 0; m < M; ++m) {
    const SubHost& o = sh[m];
    FcSubDev& d = P.s[slot_of[m]];
    // the kernels use c_m modulo N only: keep it in [0, N) so that a bin index c_m + p -
    // floor(L/2) needs one correction, not a division
    const int Ng = gh[o.g].N;
    d.L = o.L; d.Lofdm = o.Lo; d.Lact = o.Lact; d.c = ((o.c % Ng) + Ng) % Ng; d.group = o.g;
    d.L_S = o.L_S; d.L_L = o.L_L; d.L_T = o.L_T; d.S_L = o.S_L; d.n_low = o.n_low;
    d.p_lo = plo[m]; d.p_hi = phi[m];
    d.size_L = s_sizeL[m]; d.size_O = s_sizeO[m];
    d.grid_off = grid_off[m];
    d.ws_off = ws_off[m];
    d.dtx = reinterpret_cast<const float*>(base + off_dtx[m]);
    d.drx = reinterpret_cast<const float*>(base + off_drx[m]);
    d.lcp = reinterpret_cast<const int*>(base + off_lcp[m]);
    d.soff = reinterpret_cast<const int*>(base + off_soff[m]);
    d.time_tx_off = (int)t_tx_off[m];
    d.time_rx_off = (int)t_rx_off[m];
  }
  std::memcpy(blob.bytes.data() + off_plan, &P, sizeof(P));
  if (upload) {
    cudaError_t e = cudaMemcpy(base, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy of plan tables");
  }

  pl->d_plan = reinterpret_cast<FcPlanDev*>(base + off_plan);
  pl->d_jobs = reinterpret_cast<FcJob*>(base + off_jobs);
  pl->n_jobs = n_jobs;
  pl->splits = splits;
  for (size_t i = 0; i < splits.size(); ++i) {
    pl->tx_chunks.push_back(reinterpret_cast<const FcChunk*>(base + off_txc[i]));
    pl->rx_chunks.push_back(reinterpret_cast<const FcChunk*>(base + off_rxc[i]));
  }
  pl->tx_nchunks = ntx;
  pl->rx_nchunks = nrx;
  pl->warp_path = warp_ok;
  pl->warp_weight_floats = 0;
  if (warp_ok)
    for (int g = 0; g < G; ++g) pl->warp_weight_floats += sh[gh[g].subs[0]].L;
  pl->cont_warp_tx = cont_warp && geo->scheme_tx == FC_OLS;
  pl->cont_warp_rx = cont_warp && geo->scheme_rx == FC_OLS;
  pl->tc_tx = tc_tx;
  pl->tc_rx = tc_rx;
  pl->tc_ofdm = tc_tx && sh[0].Lo == 4096 && !io_time;
  if (tc_tx) {
    pl->d_dft64 = base + off_dft;
    pl->d_err = reinterpret_cast<int*>(base + off_err);
  }
  if (warp_ok) {
    pl->d_wjobs = reinterpret_cast<FcJob*>(base + off_wjobs);
    pl->n_wjobs_big = n_big;
    pl->n_wjobs_init = n_init;
    pl->d_wpjobs = reinterpret_cast<FcJob*>(base + off_wtx);
    pl->n_wpjobs = n_wtx;
    pl->d_wrxjobs = reinterpret_cast<FcJob*>(base + off_wrx);
    pl->n_wrxjobs = n_wrx;
  }
  return FC_OK;
}

std::once_flag g_smem_once[64];

size_t pick_split(const fc_plan* pl, int n_streams) {
  const long long want = 2LL * pl->num_sms;
  size_t k = 0;
  while (k + 1 < pl->splits.size() && (long long)n_streams * pl->splits[k] < want) ++k;
  return k;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_io(const fc_plan* plan, int32_t n_streams, const void* in, const void* out, const void* ws,
             size_t ws_bytes) {
  if (!plan) return fail(FC_ERR_INVALID, "plan is NULL");
  if (n_streams < 0) return fail(FC_ERR_INVALID, "n_streams < 0");
  if (n_streams == 0) return FC_OK;
  if (!in || !out) return fail(FC_ERR_INVALID, "input or output pointer is NULL");
  if (((uintptr_t)in | (uintptr_t)out) & (uintptr_t)(plan->sizes.sample_bytes - 1))
    return fail(FC_ERR_INVALID, "buffers must be aligned to the sample size (8 bytes, 4 with FC_FLAG_IO_BF16)");
  const long long need = (long long)n_streams * plan->sizes.workspace_per_stream;
  if (need > 0) {
    if (!ws || ws_bytes < (size_t)need) return fail(FC_ERR_INVALID, "workspace missing or too small");
    if ((uintptr_t)ws & 15) return fail(FC_ERR_INVALID, "workspace must be 16-byte aligned");
  }
  if ((long long)n_streams * plan->tx_nchunks.back() > 0x7fffffffLL) return fail(FC_ERR_INVALID, "too many streams");
  return FC_OK;
}

// Launch shape for this call: the autotuned or set choice if there is one
Choice choose(const fc_plan* pl, int n_streams, int dir) {
  {
    std::lock_guard<std::mutex> lock(pl->tune_mu);
    auto it = pl->tuned.find({n_streams, dir});
    if (it != pl->tuned.end()) return it->second;
  }
  Choice c;
  c.split = (int)pick_split(pl, n_streams);
  return c;
}

// Generic-kernel set of a call launching n_ctas CTAs per kernel: the chosen one, else
// 128-thread CTAs where the call fills four per SM, else 256-thread CTAs where they fit,
// else 512. (Measured: 128-thread CTAs lose on calls too small to fill the GPU, such as a
// batch's one-stream calls on concurrent lanes; 256-thread CTAs win even there, and for
// one-stream serving calls.)
const FcGenKernels& gen_for(const fc_plan* pl, long long n_ctas, int set) {
  if (set >= 0 && set < 3 && pl->gen_fits[set]) return *pl->gen[set];
  if (pl->gen_fits[2] && n_ctas >= 4LL * pl->num_sms) return *pl->gen[2];
  if (pl->gen_fits[1]) return *pl->gen[1];
  return *pl->gen[0];
}

// io: FC_IO_* bits of this call's input and output; the one-warp kernels take complex64
// and complex BF16, the tensor-core kernels complex64 only (a plan with FC_FLAG_IO_BF16
// never selects them)
cudaError_t launch_tx(const fc_plan* plan, int n_streams, const void* in, void* out, float2* workspace,
                      cudaStream_t st, Choice c, int io) {
  const size_t k = (size_t)c.split;
  const FcGenKernels& gen = gen_for(plan, (long long)n_streams * plan->tx_nchunks[k], c.set);
  const float2* grid = (const float2*)in;
  float2* wave = (float2*)out;
  if (plan->warp_path && !c.generic) {
    // float4 reductions of the warp kernel need a 16-byte aligned complex64 waveform: the
    // output itself, or for a BF16 output the workspace (frame_len samples a stream)
    const bool out16 = (io & FC_IO_OUT_BF16) != 0;
    float2* acc = out16 ? workspace : wave;
    if (acc && ((uintptr_t)acc & 15) == 0) {
      // complex64 input: the N = 1024 symbols in pairs; BF16 input: one symbol a job
      const bool in16 = (io & FC_IO_IN_BF16) != 0;
      cudaError_t e = fc_launch_tx_sync_warp(plan->d_plan, in16 ? plan->d_wjobs : plan->d_wpjobs,
                                             in16 ? plan->n_jobs : plan->n_wpjobs, plan->n_wjobs_init,
                                             plan->n_wjobs_big, n_streams,
                                             plan->h.frame_len, plan->warp_weight_floats, in, in16, acc,
                                             plan->num_sms, st);
      if (e == cudaSuccess && out16)
        e = fc_launch_to_bf16(acc, out, (long long)n_streams * plan->h.frame_len, plan->num_sms, st);
      return e;
    }
  }
  if (plan->h.mode == FC_SYMBOL_SYNC)
    return gen.tx_sync(plan->d_plan, plan->d_jobs, plan->tx_chunks[k], plan->tx_nchunks[k], n_streams, in,
                              out, io, plan->smem_tx, st);
  if (plan->cont_warp_tx && !c.generic)
    return fc_launch_tx_cont_warp(plan->d_plan, n_streams, plan->h.g[0].B, plan->h.g[0].R, in, workspace, out, io,
                                  plan->num_sms, st);
  if (plan->tc_tx && !c.generic && io == 0) {
    const int R = plan->h.g[0].R;
    cudaError_t e = plan->tc_ofdm ? fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_OFDM_MOD, n_streams,
                                                 plan->h.g[0].B, grid, nullptr, workspace, plan->d_err,
                                                 plan->num_sms, st, plan->tc_first_wait)
                                  : gen.ofdm_mod(plan->d_plan, plan->syms_per_stream, n_streams, grid,
                                                        workspace, 0, plan->smem_ofdm, st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(wave, 0, (size_t)n_streams * plan->h.frame_len * sizeof(float2), st);
    if (e == cudaSuccess)
      e = fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_TX_FFT, n_streams, R, nullptr, nullptr, workspace,
                       plan->d_err, plan->num_sms, st, plan->tc_first_wait);
    if (e == cudaSuccess)
      e = fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_TX_IFFT, n_streams, R, nullptr, wave, workspace,
                       plan->d_err, plan->num_sms, st, plan->tc_first_wait);
    return e;
  }
  cudaError_t e = gen.ofdm_mod(plan->d_plan, plan->syms_per_stream, n_streams, in, workspace, io,
                                      plan->smem_ofdm, st);
  if (e == cudaSuccess)
    e = gen.tx_cont(plan->d_plan, plan->d_jobs, plan->tx_chunks[k], plan->tx_nchunks[k], n_streams, workspace,
                           out, io, plan->smem_tx, st);
  return e;
}

cudaError_t launch_rx(const fc_plan* plan, int n_streams, const void* in, void* out, float2* workspace,
                      cudaStream_t st, Choice c, int io) {
  const size_t k = (size_t)c.split;
  const FcGenKernels& gen = gen_for(plan, (long long)n_streams * plan->rx_nchunks[k], c.set);
  const float2* wave = (const float2*)in;
  float2* grid = (float2*)out;
  if (plan->warp_path && !c.generic) {
    // a BF16 waveform is widened into the workspace (frame_len samples a stream) first
    const void* x = in;
    if ((io & FC_IO_IN_BF16) && workspace && ((uintptr_t)workspace & 15) == 0) {
      cudaError_t e = fc_launch_from_bf16(in, workspace, (long long)n_streams * plan->h.frame_len, plan->num_sms, st);
      if (e != cudaSuccess) return e;
      x = workspace;
    }
    if (!(io & FC_IO_IN_BF16) || x != in)
      return fc_launch_rx_sync_warp(plan->d_plan, plan->d_wrxjobs, plan->n_wrxjobs, plan->n_wjobs_big, n_streams,
                                    plan->warp_weight_floats, plan->h.scheme_rx, plan->h.flags, x, out,
                                    io & FC_IO_OUT_BF16, plan->num_sms, st);
  }
  if (plan->h.mode == FC_SYMBOL_SYNC)
    return gen.rx_sync(plan->d_plan, plan->d_jobs, plan->rx_chunks[k], plan->rx_nchunks[k], n_streams, in,
                              out, io, plan->smem_rx, st);
  if (plan->cont_warp_rx && !c.generic)
    return fc_launch_rx_cont_warp(plan->d_plan, n_streams, plan->h.g[0].B, plan->h.g[0].R, in, workspace, out, io,
                                  plan->num_sms, st);
  if (plan->tc_rx && !c.generic && io == 0) {
    const int R = plan->h.g[0].R;
    cudaError_t e = fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_RX_FFT, n_streams, R, wave, nullptr, workspace,
                                 plan->d_err, plan->num_sms, st, plan->tc_first_wait);
    if (e == cudaSuccess)
      e = fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_RX_IFFT, n_streams, R, nullptr, nullptr, workspace,
                       plan->d_err, plan->num_sms, st, plan->tc_first_wait);
    if (e == cudaSuccess)
      e = plan->tc_ofdm ? fc_launch_tc(plan->d_plan, plan->d_dft64, FC_TC_OFDM_DEMOD, n_streams, plan->h.g[0].B,
                                       nullptr, grid, workspace, plan->d_err, plan->num_sms, st, plan->tc_first_wait)
                        : gen.ofdm_demod(plan->d_plan, plan->syms_per_stream, n_streams, workspace, grid,
                                                0, plan->smem_ofdm, st);
    return e;
  }
  cudaError_t e = gen.rx_cont(plan->d_plan, plan->d_jobs, plan->rx_chunks[k], plan->rx_nchunks[k], n_streams,
                                     in, workspace, io, plan->smem_rx, st);
  if (e == cudaSuccess)
    e = gen.ofdm_demod(plan->d_plan, plan->syms_per_stream, n_streams, workspace, out, io, plan->smem_ofdm,
                              st);
  return e;
}

}  // namespace

int fc_internal_fail(int code, const char* msg) { return fail(code, msg); }

int fc_internal_plan_device(const fc_plan* plan) { return plan ? plan->device : -1; }

int fc_internal_num_sms(const fc_plan* plan) { return plan ? plan->num_sms : 0; }

int fc_internal_io(const fc_plan* plan) { return plan ? plan->io : 0; }

// persistent launches fill every SM: the smallest CTAs that fit
const FcGenKernels& fc_internal_gen(const fc_plan* plan) {
  return *plan->gen[plan->gen_fits[2] ? 2 : (plan->gen_fits[1] ? 1 : 0)];
}

int fc_internal_frame(const fc_plan* plan, int dir, int n_streams, const void* in, void* out, void* workspace,
                      size_t workspace_bytes, void* stream, int io) {
  int rc = check_io(plan, n_streams, in, out, workspace, workspace_bytes);
  if (rc != FC_OK || n_streams == 0) return rc;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return fail(FC_ERR_CUDA, "cudaSetDevice failed");
  const Choice c = choose(plan, n_streams, dir);
  const cudaError_t e = dir == FC_TX ? launch_tx(plan, n_streams, in, out, (float2*)workspace, (cudaStream_t)stream, c, io)
                                     : launch_rx(plan, n_streams, in, out, (float2*)workspace, (cudaStream_t)stream, c, io);
  return e == cudaSuccess ? FC_OK : cuda_fail(e, dir == FC_TX ? "TX kernel launch" : "RX kernel launch");
}

bool fc_internal_sync_work(const fc_plan* plan, int dir, int n_streams, const void* in, void* out,
                           std::vector<FcWork>& work, size_t* smem) {
  if (!plan || plan->h.mode != FC_SYMBOL_SYNC || n_streams < 1) return false;
  const Choice c = choose(plan, n_streams, dir);
  if (plan->warp_path && !c.generic) return false;       // the specialised kernels run this call
  const size_t k = (size_t)c.split;
  const FcChunk* chunks = dir == FC_TX ? plan->tx_chunks[k] : plan->rx_chunks[k];
  const int n_chunks = dir == FC_TX ? plan->tx_nchunks[k] : plan->rx_nchunks[k];
  for (int s = 0; s < n_streams; ++s)
    for (int ch = 0; ch < n_chunks; ++ch)
      work.push_back(FcWork{plan->d_plan, plan->d_jobs, chunks + ch, in, out, s, plan->io});
  *smem = dir == FC_TX ? plan->smem_tx : plan->smem_rx;
  return true;
}

bool fc_internal_sync_work_generic(const fc_plan* plan, int dir, int n_streams, const void* in, void* out,
                                   int want_chunks, std::vector<FcWork>& work, size_t* smem) {
  if (!plan || plan->h.mode != FC_SYMBOL_SYNC || n_streams < 1 || plan->io != 0) return false;
  if (plan->h.flags & FC_FLAG_IO_TIME) return false;
  size_t k = 0;
  while (k + 1 < plan->splits.size() && plan->splits[k] < want_chunks) ++k;
  const FcChunk* chunks = dir == FC_TX ? plan->tx_chunks[k] : plan->rx_chunks[k];
  const int n_chunks = dir == FC_TX ? plan->tx_nchunks[k] : plan->rx_nchunks[k];
  for (int s = 0; s < n_streams; ++s)
    for (int ch = 0; ch < n_chunks; ++ch)
      work.push_back(FcWork{plan->d_plan, plan->d_jobs, chunks + ch, in, out, s, 0});
  *smem = dir == FC_TX ? plan->smem_tx : plan->smem_rx;
  return true;
}

extern "C" {

int fc_plan_create(fc_plan** out, const fc_geometry* geometry, int32_t device) {
  FcRange nvtx_range(__func__);
  if (!out) return fail(FC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev || device >= 64) return fail(FC_ERR_INVALID, "device out of range");
  DeviceGuard dg(device);
  if (!dg.ok) return fail(FC_ERR_CUDA, "cudaSetDevice failed");
  fc_plan* pl = new fc_plan();
  pl->device = device;
  e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  const size_t reserve = sizeof(FcPlanDev) + 256;   // static shared memory of the kernels
  pl->smem_cap = (size_t)optin > reserve ? (size_t)optin - reserve : 0;
  int per_sm = 0;
  e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  pl->smem_sm = (size_t)per_sm;
  cudaError_t se = cudaSuccess;
  std::call_once(g_smem_once[device], [&] {
    se = fc_gen_kernels_512().set_smem_limits(pl->smem_cap);
    if (se == cudaSuccess) se = fc_gen_kernels_256().set_smem_limits(pl->smem_cap);
    if (se == cudaSuccess) se = fc_gen_kernels_128().set_smem_limits(pl->smem_cap);
    if (se == cudaSuccess) se = fc_set_warp_smem_limits();
    if (se == cudaSuccess) se = fc_set_tc_smem_limits();
  });
  if (se != cudaSuccess) {
    delete pl;
    return cuda_fail(se, "cudaFuncSetAttribute");
  }
  const int rc = build_plan(pl, geometry, true);
  if (rc != FC_OK) {
    if (pl->d_mem) cudaFree(pl->d_mem);
    delete pl;
    return rc;
  }
  // Reserve the allocation-free TX entry point's device array now, at set-up, rather
  // than at its first call. A failure here does not fail the plan (most callers never
  // use that entry point); fc_tx_synthesize_static retries and reports it.
  fc_internal_static_resolve(device);
  *out = pl;
  return FC_OK;
}

int fc_geometry_check(const fc_geometry* geometry, fc_sizes* out) {
  fc_plan tmp;
  const int rc = build_plan(&tmp, geometry, false);
  if (rc == FC_OK && out) *out = tmp.sizes;
  return rc;
}

int fc_query(const fc_plan* plan, fc_sizes* out) {
  if (!plan || !out) return fail(FC_ERR_INVALID, "NULL argument");
  *out = plan->sizes;
  return FC_OK;
}

int fc_tx_synthesize(const fc_plan* plan, int32_t n_streams, const void* grid_in, void* wave_out, void* workspace,
                     size_t workspace_bytes, void* stream) {
  FcRange nvtx_range(__func__);
  return fc_internal_frame(plan, FC_TX, n_streams, grid_in, wave_out, workspace, workspace_bytes, stream,
                           plan ? plan->io : 0);
}

int fc_rx_analyze(const fc_plan* plan, int32_t n_streams, const void* wave_in, void* grid_out, void* workspace,
                  size_t workspace_bytes, void* stream) {
  FcRange nvtx_range(__func__);
  return fc_internal_frame(plan, FC_RX, n_streams, wave_in, grid_out, workspace, workspace_bytes, stream,
                           plan ? plan->io : 0);
}

int fc_plan_autotune(fc_plan* plan, int32_t n_streams, int32_t reps, void* stream) {
  FcRange nvtx_range(__func__);
  if (!plan) return fail(FC_ERR_INVALID, "plan is NULL");
  if (n_streams < 1 || reps < 1) return fail(FC_ERR_INVALID, "need n_streams >= 1 and reps >= 1");
  DeviceGuard dg(plan->device);
  if (!dg.ok) return fail(FC_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  const fc_sizes& z = plan->sizes;
  // complex64-sized buffers also hold a BF16 call's samples; grid or time-domain I/O
  const size_t n_grid = (size_t)n_streams * (size_t)std::max(z.tx_in_len, z.rx_out_len);
  const size_t n_wave = (size_t)n_streams * z.wave_len;
  const size_t ws_bytes = (size_t)n_streams * z.workspace_per_stream;
  // tuning buffers (zeros: the kernels' time does not depend on the values)
  unsigned char* mem = nullptr;
  const size_t bytes = (n_grid + n_wave) * sizeof(float2) + ws_bytes + 256;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(FC_ERR_NOMEM, "autotune buffers")
                                                              : cuda_fail(e, "cudaMalloc");
  e = cudaMemsetAsync(mem, 0, bytes, st);
  float2* grid = (float2*)mem;
  float2* wave = grid + n_grid;
  float2* ws = (float2*)(((uintptr_t)(wave + n_wave) + 255) & ~(uintptr_t)255);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  Choice best[2];
  for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir) {
    float best_ms = 1e30f;
    const bool special = dir == FC_TX ? (plan->warp_path || plan->tc_tx || plan->cont_warp_tx)
                                      : (plan->warp_path || plan->tc_rx || plan->cont_warp_rx);
    // candidates: every split with the specialised kernels (where they apply), and every
    // split on every generic-kernel set that fits
    std::vector<Choice> cand;
    for (int k = 0; k < (int)plan->splits.size(); ++k) {
      // the one-warp-per-symbol kernels deal all streams' jobs to the GPU whatever the
      // split; the tensor-core passes take no split either
      if (special && k == 0) cand.push_back(Choice{k, 0, -1});
      for (int set = 0; set < 3; ++set)
        if (plan->gen_fits[set]) cand.push_back(Choice{k, special ? 1 : 0, set});
    }
    for (const Choice& c : cand) {
      if (e != cudaSuccess) break;
      auto run = [&]() {
        return dir == FC_TX ? launch_tx(plan, n_streams, grid, wave, ws, st, c, plan->io)
                            : launch_rx(plan, n_streams, wave, grid, ws, st, c, plan->io);
      };
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best[dir] = c;
      }
    }
  }
  // Radix schedules of the generic kernels' transforms (the plan's device table, read by
  // every generic launch): per transform size in turn, each candidate schedule is timed
  // on the directions whose best launch shape runs the generic kernels, and the fastest
  // is kept (the specialised and tensor-core kernels have fixed transforms of their own).
  bool gen_dir[2];
  for (int dir = 0; dir < 2; ++dir) {
    const bool special = dir == FC_TX ? (plan->warp_path || plan->tc_tx || plan->cont_warp_tx)
                                      : (plan->warp_path || plan->tc_rx || plan->cont_warp_rx);
    gen_dir[dir] = !special || best[dir].generic;
  }
  for (int i = 0; i < plan->h.n_sizes && e == cudaSuccess && (gen_dir[0] || gen_dir[1]); ++i) {
    FcSize& z = plan->h.sz[i];
    const auto cands = radix_candidates(z.n);
    if (cands.size() < 2) continue;
    float best_ms = 1e30f;
    std::vector<unsigned char> keep(z.radix, z.radix + z.npass);
    for (const auto& r : cands) {
      if (e != cudaSuccess) break;
      z.npass = (int)r.size();
      std::copy(r.begin(), r.end(), z.radix);
      e = cudaMemcpy(plan->d_plan, &plan->h, sizeof(FcPlanDev), cudaMemcpyHostToDevice);
      auto run = [&]() {
        cudaError_t x = cudaSuccess;
        if (gen_dir[FC_TX]) x = launch_tx(plan, n_streams, grid, wave, ws, st, best[FC_TX], plan->io);
        if (x == cudaSuccess && gen_dir[FC_RX]) x = launch_rx(plan, n_streams, wave, grid, ws, st, best[FC_RX], plan->io);
        return x;
      };
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
      for (int r2 = 0; r2 < reps && e == cudaSuccess; ++r2) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        keep = r;
      }
    }
    z.npass = (int)keep.size();
    std::copy(keep.begin(), keep.end(), z.radix);
    if (e == cudaSuccess) e = cudaMemcpy(plan->d_plan, &plan->h, sizeof(FcPlanDev), cudaMemcpyHostToDevice);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  cudaStreamSynchronize(st);
  cudaFree(mem);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  std::lock_guard<std::mutex> lock(plan->tune_mu);
  plan->tuned[{n_streams, FC_TX}] = best[FC_TX];
  plan->tuned[{n_streams, FC_RX}] = best[FC_RX];
  return FC_OK;
}

int fc_plan_radices(const fc_plan* plan, int32_t n, int32_t* radices, int32_t* n_passes) {
  if (!plan || !radices || !n_passes) return fail(FC_ERR_INVALID, "NULL argument");
  for (int i = 0; i < plan->h.n_sizes; ++i) {
    const FcSize& z = plan->h.sz[i];
    if (z.n != n) continue;
    *n_passes = z.npass;
    for (int k = 0; k < z.npass; ++k) radices[k] = z.radix[k];
    return FC_OK;
  }
  return fail(FC_ERR_INVALID, "the plan has no transform of that size");
}

int fc_plan_set_choice(fc_plan* plan, int32_t n_streams, int32_t direction, int32_t chunks_per_stream,
                       int32_t generic_kernels) {
  if (!plan || (direction != FC_TX && direction != FC_RX) || n_streams < 1 ||
      (generic_kernels != 0 && generic_kernels != 1))
    return fail(FC_ERR_INVALID, "bad plan, direction, n_streams or generic_kernels");
  const auto it = std::find(plan->splits.begin(), plan->splits.end(), (int)chunks_per_stream);
  if (it == plan->splits.end()) return fail(FC_ERR_INVALID, "chunks_per_stream is not one of the plan's splits");
  std::lock_guard<std::mutex> lock(plan->tune_mu);
  plan->tuned[{n_streams, direction}] = Choice{(int)(it - plan->splits.begin()), (int)generic_kernels, -1};
  return FC_OK;
}

int fc_plan_choice(const fc_plan* plan, int32_t n_streams, int32_t direction, int32_t* chunks_per_stream,
                   int32_t* generic_kernels) {
  if (!plan || (direction != FC_TX && direction != FC_RX) || n_streams < 1)
    return fail(FC_ERR_INVALID, "bad plan, direction or n_streams");
  const Choice c = choose(plan, n_streams, direction);
  if (chunks_per_stream) *chunks_per_stream = plan->splits[c.split];
  const bool special = direction == FC_TX ? (plan->warp_path || plan->tc_tx || plan->cont_warp_tx)
                                            : (plan->warp_path || plan->tc_rx || plan->cont_warp_rx);
  if (generic_kernels) *generic_kernels = (special && !c.generic) ? 0 : 1;
  return FC_OK;
}

int fc_plan_device_status(const fc_plan* plan) {
  if (!plan) return fail(FC_ERR_INVALID, "plan is NULL");
  if (!plan->d_err) return FC_OK;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return fail(FC_ERR_CUDA, "cudaSetDevice failed");
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(plan->d_err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  return v ? fail(FC_ERR_TIMEOUT, "a tensor-core kernel gave up waiting for its MMAs") : FC_OK;
}

int fc_plan_set_first_wait_limit(fc_plan* plan, uint32_t polls) {
  if (!plan) return fail(FC_ERR_INVALID, "plan is NULL");
  plan->tc_first_wait = polls;
  return FC_OK;
}

void fc_plan_destroy(fc_plan* plan) {
  if (!plan) return;
  {
    DeviceGuard dg(plan->device);
    if (plan->d_mem) cudaFree(plan->d_mem);
  }
  delete plan;
}

const char* fc_status_string(int status) {
  switch (status) {
    case FC_OK: return "FC_OK";
    case FC_ERR_INVALID: return "FC_ERR_INVALID: invalid geometry or argument";
    case FC_ERR_UNSUPPORTED: return "FC_ERR_UNSUPPORTED: size or layout the library has no kernel for";
    case FC_ERR_NOMEM: return "FC_ERR_NOMEM: device allocation failed";
    case FC_ERR_CUDA: return "FC_ERR_CUDA: CUDA runtime error";
    case FC_ERR_TIMEOUT: return "FC_ERR_TIMEOUT: bounded device wait expired";
    default: return "unknown status";
  }
}

const char* fc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
