// C ABI of libclusterspec (declared in include/cs.h): context, tables, workspace layout and
// the host-side drivers of H.X, the Chebyshev filter, Cholesky-QR, Rayleigh-Ritz, the
// Lanczos bound and the ChFSI loop. Every numerical step runs in this library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cs_internal.h"
#include "df64.cuh"
#include "hx_kernels.cuh"
#include "kb_tc.h"

using namespace cs;

namespace {

thread_local std::string g_init_error;

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t G, Yalt, X32, Wkb, kbZ, HX, tmp, part, small, lanV, status, HXr, chw, oz, wd, kbtc, wa,
      total;
};

constexpr int kMaxLanczos = 64;
// largest degree of the residual-form filter (its weight table is sized for it)
constexpr int kMaxRitzDegree = 64;

Layout layout(const cs_ctx* c, int n_s, cs_precision prec) {
  const HostTables& T = c->host;
  const size_t d = (size_t)T.d, ns = (size_t)n_s, L2 = (size_t)T.L * T.L;
  const size_t np = (size_t)c->n_p;
  Layout o{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += al256(bytes);
    return at;
  };
  o.G = take((size_t)T.n_r * L2 * ns * 8);
  o.Yalt = take(d * ns * 8);
  o.Wkb = take(np * ns * 8);
  o.kbZ = take(np ? d * ns * 8 : 0);
  o.HX = take(d * ns * 8);
  o.tmp = take(d * ns * 8);
  size_t part = std::max(gram_partial_elems(T.d, n_s, n_s),
                         gram_partial_elems(T.d, kMaxLanczos + 1, 1));
  if (np) part = std::max(part, gram_partial_elems(T.d, (int)np, n_s));
  o.part = take(part * 8);
  // small matrices: Gram / Rayleigh-Ritz matrix, rotation, and the eigensolver scratch
  // (8 m^2 + 3 m + 4 doubles), with m = max(n_s, Lanczos size)
  const size_t mm = std::max<size_t>(ns, kMaxLanczos + 2);
  o.small = take((12 * mm * mm + 32 * mm + 4096) * 8);
  o.lanV = take(d * (kMaxLanczos + 2) * 8);
  o.status = take(64 * sizeof(int));
  // H X of the current Ritz vectors, kept between ChFSI iterations (residual-form filter)
  o.HXr = take(d * ns * 8);
  // weights s_i(theta_j) of the residual-form filter: FP64 table and one in the block type
  o.chw = take((size_t)(kMaxRitzDegree + 1) * ns * 16);
  // split operands and partial sums of the slice-product Gram matrices and rotations (and of
  // the FP64 projector pair, which takes the same arithmetic)
  size_t ozb = 0;
  if (c->dense_prec == CS_FP64_SLICED) {
    ozb = std::max(oz_gram_work_bytes(T.d, n_s, n_s, false), oz_rotate_work_bytes(T.d, n_s, n_s));
    if (np)
      ozb = std::max(ozb, std::max(oz_gram_work_bytes(T.d, (int)np, n_s, false),
                                   oz_rotate_work_bytes(T.d, (int)np, n_s)));
  }
  o.oz = take(ozb);
  // double-float intermediate of the three-pass angular block (one block of 32 states), sized
  // whenever that block is eligible, whatever the precision of the call
  o.wd = take(angular_wide_df_eligible(T.L, T.n_theta, T.n_phi)
                  ? angular_wide_df_work_bytes(T.L, T.n_r, T.n_theta)
                  : 0);
  // last, so that every other offset is the same for both precisions
  auto is_f32 = [](cs_precision p) { return p == CS_FP32 || p == CS_MIXED_BF16; };
  const bool reduced = is_f32(prec) || is_f32(c->rr_prec);
  const bool mixed = prec == CS_MIXED_BF16 || c->rr_prec == CS_MIXED_BF16;
  o.X32 = take(reduced ? d * ns * 4 : 0);
  // scratch of the tensor-core projector products (mixed precision with projectors)
  o.kbtc = take(mixed && np ? kb_tc_work_bytes(kb_tc_shape(T.d, (int)np, n_s)) : 0);
  // FP32 intermediate of the three-pass tensor-core angular block (sized whenever the block
  // is eligible, so that the choice of angular kernel never changes the workspace size)
  o.wa = take(mixed && angular_wide_eligible(T.L, T.n_theta, T.n_phi)
                  ? angular_wide_work_bytes(T.L, T.n_r, T.n_theta, n_s)
                  : 0);
  o.total = off;
  return o;
}

template <typename T>
DevTables<T>& tables(cs_ctx* c);
template <>
DevTables<double>& tables<double>(cs_ctx* c) { return c->d64; }
template <>
DevTables<float>& tables<float>(cs_ctx* c) { return c->d32; }
template <>
DevTables<df64>& tables<df64>(cs_ctx* c) { return c->ddf; }

cs_status fail(cs_ctx* c, cs_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CS_CHECK_CUDA(ctx, expr)                                                       \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, CS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Event pair around a launch while profiling is on (class cls, see cs_profile_end).
struct ProfScope {
  cs_ctx* c;
  cudaStream_t st;
  cudaEvent_t b = nullptr;
  int cls;
  static cudaEvent_t get(cs_ctx* c) {
    if (!c->event_pool.empty()) {
      cudaEvent_t e = c->event_pool.back();
      c->event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  ProfScope(cs_ctx* c_, int cls_, cudaStream_t st_) : c(c_), st(st_), cls(cls_) {
    if (c->prof) {
      cudaEvent_t a = get(c);
      b = get(c);
      cudaEventRecord(a, st);
      c->prof_recs.push_back({cls, a, b});
    }
  }
  ~ProfScope() {
    if (b) cudaEventRecord(b, st);
  }
};

#define CS_LAUNCH_CLS(ctx, cls, nk, expr)  \
  do {                                     \
    ProfScope ps_((ctx), (cls), st);       \
    CS_CHECK_CUDA(ctx, expr);              \
    (ctx)->launches += (nk);               \
  } while (0)
#define CS_LAUNCH(ctx, nk, expr) CS_LAUNCH_CLS(ctx, 3, nk, expr)
constexpr int kProfFamilies = 5;  // classes per arithmetic (see cs_ctx::prof)
template <typename T>
constexpr int prof_cls(int family) {
  return family + (std::is_same<T, float>::value ? kProfFamilies
                   : std::is_same<T, df64>::value ? 2 * kProfFamilies : 0);
}

cs_status need_device(cs_ctx* c) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) return fail(c, CS_ERR_STATE, "context has no device (created with device < 0)");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, CS_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return CS_OK;
}

template <typename T>
cs_status upload(cs_ctx* c, T** dst, const std::vector<double>& src) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  size_t bytes = std::max<size_t>(tmp.size(), 1) * sizeof(T);
  if (cudaMalloc((void**)dst, bytes) != cudaSuccess) return fail(c, CS_ERR_ALLOC, "cudaMalloc of a table failed");
  if (!tmp.empty() &&
      cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, CS_ERR_CUDA, "table upload failed");
  return CS_OK;
}

template <typename T>
void free_tables(DevTables<T>& D) {
  T** ptrs[] = {&D.rad, &D.theta, &D.trig, &D.wv, &D.wkj, &D.half_lambda, &D.pcoef, &D.h,
                &D.theta_pairs};
  for (T** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

template <typename T>
cs_status upload_tables(cs_ctx* c) {
  const HostTables& H = c->host;
  DevTables<T>& D = tables<T>(c);
  cs_status st;
  if ((st = upload<T>(c, &D.rad, H.rad)) != CS_OK) return st;
  const int rowlen = theta_row_len(H.L);
  const int rows = (H.n_theta + 1) / 2;
  std::vector<double> th(H.theta.begin(), H.theta.begin() + (size_t)rows * rowlen);
  if ((st = upload<T>(c, &D.theta, th)) != CS_OK) return st;
  const int Q = c->Q4 + 1;
  std::vector<double> trig((size_t)2 * H.L * Q);
  for (int m = 0; m < H.L; ++m)
    for (int q = 0; q < Q; ++q) {
      double ang = 2.0 * 3.14159265358979323846 * (double)((long long)m * q % H.n_phi) / H.n_phi;
      double cv = std::cos(ang), sv = std::sin(ang);
      // quarter-turn angles have exact zeros; the folded phi sums rely on them
      trig[(size_t)m * Q + q] = std::fabs(cv) < 1e-12 ? 0.0 : cv;
      trig[(size_t)(H.L + m) * Q + q] = std::fabs(sv) < 1e-12 ? 0.0 : sv;
    }
  if ((st = upload<T>(c, &D.trig, trig)) != CS_OK) return st;
  if (sizeof(T) == 4) {
    std::vector<double> tp;
    build_theta_pairs(th, trig, H.L, c->Q4, H.n_theta, tp);
    if ((st = upload<T>(c, &D.theta_pairs, tp)) != CS_OK) return st;
  }
  std::vector<double> wkj((size_t)H.n_r * H.n_theta);
  for (int k = 0; k < H.n_r; ++k)
    for (int j = 0; j < H.n_theta; ++j)
      wkj[(size_t)k * H.n_theta + j] =
          H.w_r[k] * H.w_t[j] * (2.0 * 3.14159265358979323846 / H.n_phi);
  if ((st = upload<T>(c, &D.wkj, wkj)) != CS_OK) return st;
  if ((st = upload<T>(c, &D.half_lambda, H.half_lambda)) != CS_OK) return st;
  size_t ng = (size_t)H.n_r * H.n_theta * H.n_phi;
  if (cudaMalloc((void**)&D.wv, ng * sizeof(T)) != cudaSuccess)
    return fail(c, CS_ERR_ALLOC, "cudaMalloc of W*V failed");
  return CS_OK;
}

// ------------------------------------------------------------------ H.X core
// out = epilogue(1/2 Lambda X + Z (+ kb)); see Epilogue in hx_kernels.cuh
template <typename T>
cs_status hx_core(cs_ctx* c, int n_s, const T* X, long long ldx, T* out, long long ldo, int mode,
                  double cA, double cB, double csh, const T* Yprev, char* work, cudaStream_t st,
                  bool tc = false, const T* src = nullptr, const T* src_w = nullptr,
                  const T* kb_in = nullptr) {
  const HostTables& H = c->host;
  DevTables<T>& D = tables<T>(c);
  const Layout lay = layout(c, n_s, CS_FP64);
  T* G = reinterpret_cast<T*>(work + lay.G);
  const T* kb = kb_in;  // a projector term the caller formed already (double-float apply)
  if (kb_in) {
  } else if constexpr (std::is_same<T, df64>::value) {
    if (c->n_p > 0) return fail(c, CS_ERR_STATE, "CS_DF64 does not apply projectors");
  } else if (c->n_p > 0) {
    // kb = P diag(h) P^T X  (Sec. 2.3.2: a pair of matrix products)
    T* kbZ = reinterpret_cast<T*>(work + lay.kbZ);
    if (tc) {
      const Layout lm = layout(c, n_s, CS_MIXED_BF16);
      const KbTcShape ks = kb_tc_shape(H.d, c->n_p, n_s);
      int nl = 0;
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 4,
                    launch_kb_tc(c->kb_tabA, c->kb_tabB, ks, reinterpret_cast<const float*>(X),
                                 ldx, c->d32.h, reinterpret_cast<float*>(kbZ), H.d,
                                 work + lm.kbtc, c->dev_err, st, &nl));
    } else if (std::is_same<T, double>::value && c->dense_prec == CS_FP64_SLICED) {
      // FP64 pair as exact slice products on the tensor cores (the dense steps' arithmetic)
      double* Wkb = reinterpret_cast<double*>(work + lay.Wkb);
      const double* Xd = reinterpret_cast<const double*>(X);
      double* Zd = reinterpret_cast<double*>(kbZ);
      void* oz = work + lay.oz;
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 4,
                    launch_oz_gram(c->d64.pcoef, H.d, Xd, ldx, H.d, c->n_p, n_s, Wkb, c->n_p, oz,
                                   c->dev_err, st));
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 1,
                    launch_scale_rows<double>(Wkb, c->n_p, n_s, c->n_p, c->d64.h, st));
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 4,
                    launch_oz_rotate(c->d64.pcoef, H.d, Wkb, c->n_p, H.d, c->n_p, n_s, Zd, H.d,
                                     oz, c->dev_err, st));
    } else {
      T* Wkb = reinterpret_cast<T*>(work + lay.Wkb);
      T* part = reinterpret_cast<T*>(work + lay.part);
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 2,
                    launch_gram<T>(D.pcoef, H.d, X, ldx, H.d, c->n_p, n_s, Wkb, c->n_p, part, st));
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 1, launch_scale_rows<T>(Wkb, c->n_p, n_s, c->n_p, D.h, st));
      CS_LAUNCH_CLS(c, prof_cls<T>(4), 1,
                    launch_gemm_nn<T>(D.pcoef, H.d, Wkb, c->n_p, H.d, c->n_p, n_s, 1.0, 0.0, kbZ,
                                      H.d, st));
    }
    kb = kbZ;
  }
  TcTables tt;
  tt.synth = c->tc_synth;
  tt.anal = c->tc_anal;
  tt.rows_synth = c->tc_rows_synth;
  tt.kpad_synth = c->tc_kpad_synth;
  tt.rows_anal = c->tc_rows_anal;
  tt.kpad_anal = c->tc_kpad_anal;
  if (tc && !std::is_same<T, float>::value)
    return fail(c, CS_ERR_ARG, "tensor-core path needs float blocks");
  // radial dimensions above the MMA's N limit take the FP32 tiles
  const bool tc_rad = tc && tc_radial_fits(H);
  if (tc_rad) {
    CS_LAUNCH_CLS(c, prof_cls<T>(0), 1, launch_tc_radial_synth(tt, H, reinterpret_cast<const float*>(X), ldx,
                                                  reinterpret_cast<float*>(G), n_s, c->dev_err,
                                                  st));
  } else {
    CS_LAUNCH_CLS(c, prof_cls<T>(0), 1, launch_radial_synth<T>(X, ldx, G, D.rad, H.L, H.N, H.n_r, n_s, st));
  }
  AngArgs<T> a{H.L, H.n_r, H.n_theta, H.n_phi, c->Q4, n_s, D.theta, D.trig, D.wv, D.wkj,
               D.theta_pairs};
  bool ang_done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (tc && c->wide_tab &&
        angular_wide_enabled(H.L, H.n_theta, H.n_phi, c->tc_phi != nullptr)) {
      const Layout lw = layout(c, n_s, CS_MIXED_BF16);
      CS_LAUNCH_CLS(c, prof_cls<T>(1), 3,
                    launch_angular_wide(a, c->wide_tab, G, reinterpret_cast<float*>(work + lw.wa),
                                        c->dev_err, st));
      ang_done = true;
    } else if (tc && c->tc_phi && angular_tc_enabled()) {
      CS_LAUNCH_CLS(c, prof_cls<T>(1), 1, launch_angular_tc(a, c->tc_phi, G, c->dev_err, st));
      ang_done = true;
    }
  }
  if constexpr (std::is_same<T, df64>::value) {
    if (angular_wide_df_enabled(H.L, H.n_theta, H.n_phi, c->Q4)) {
      const int nblk = (n_s + 31) / 32;
      CS_LAUNCH_CLS(c, prof_cls<T>(1), 3 * nblk,
                    launch_angular_wide_df(a, G, reinterpret_cast<df64*>(work + lay.wd), st));
      ang_done = true;
    }
  }
  if (!ang_done)
    CS_LAUNCH_CLS(c, prof_cls<T>(1), 1, launch_angular<T>(a, ANG_FULL, G, nullptr, nullptr, st));
  Epilogue<T> ep;
  ep.mode = mode;
  ep.out = out;
  ep.X = X;
  ep.ld = ldx;
  ep.ld_out = ldo;
  ep.Yprev = Yprev;
  ep.half_lambda = D.half_lambda;
  ep.kb = kb;
  ep.kb_ld = H.d;
  ep.cA = (T)cA;
  ep.cB = (T)cB;
  ep.cshift = (T)csh;
  ep.src = src;
  ep.src_w = src_w;
  ep.src_ld = H.d;
  if (tc_rad) {
    CS_LAUNCH_CLS(c, prof_cls<T>(2), 1, launch_tc_radial_anal(tt, H, reinterpret_cast<const float*>(G), n_s,
                                                 *reinterpret_cast<const Epilogue<float>*>(&ep),
                                                 c->dev_err, st));
  } else {
    CS_LAUNCH_CLS(c, prof_cls<T>(2), 1, launch_radial_anal<T>(G, D.rad, H.L, H.N, H.n_r, n_s, ep, st));
  }
  return CS_OK;
}

// H X in double-float for an FP64 block X (ld), product widened into HX (ldh); the block is
// split into `Xd`, the product formed in `Yd` (both d x n_s double-float, ld d). With projectors
// (only with CS_FP64_SLICED dense products) their term is formed first from the FP64 block as
// exact slice products, converted to double-float in place and handed to the epilogue.
cs_status hx_df64_from_fp64(cs_ctx* c, int n_s, const double* X, long long ld, double* HX,
                            long long ldh, df64* Xd, df64* Yd, char* work, cudaStream_t st);

template <typename T>
cs_status cheb_core(cs_ctx* c, int n_s, T* X, long long ld, int degree, double a, double b,
                    double a0, char* work, cudaStream_t st, bool tc = false) {
  const HostTables& H = c->host;
  const Layout lay = layout(c, n_s, CS_FP64);
  T* alt = reinterpret_cast<T*>(work + lay.Yalt);
  const long long lda = H.d;
  const double cc = 0.5 * (a + b), e = 0.5 * (b - a);
  const double s1 = e / (a0 - cc);
  // Y_1 = (sigma_1/e)(H - c) Y_0 into alt
  cs_status r = hx_core<T>(c, n_s, X, ld, alt, lda, EP_CHEB, s1 / e, 0.0, cc, nullptr, work, st, tc);
  if (r != CS_OK) return r;
  T* prev = X;
  long long ldp = ld;
  T* cur = alt;
  long long ldc = lda;
  double sig = s1;
  for (int i = 1; i < degree; ++i) {
    double sn = 1.0 / (2.0 / s1 - sig);
    // Y_{i+1} = (2 sn/e)(H - c) Y_i - sig sn Y_{i-1}, written over Y_{i-1}
    r = hx_core<T>(c, n_s, cur, ldc, prev, ldp, EP_CHEB, 2.0 * sn / e, sig * sn, cc, prev, work, st,
                   tc);
    if (r != CS_OK) return r;
    std::swap(prev, cur);
    std::swap(ldp, ldc);
    sig = sn;
  }
  if (cur != X) CS_LAUNCH(c, 1, launch_copy_block<T>(cur, ldc, X, ld, H.d, n_s, st));
  return CS_OK;
}

// Residual form of the filter (cheb_ritz.cu): X <- X s_m(Theta) + D_m for Ritz vectors X
// (FP64), their H X (FP64) and Ritz values theta (device). The deviation D runs through the
// recurrence in the block type T, with R = H X - X Theta as the source of each step: degree - 1
// H.X products (D_1 needs none). Buffers: R in tmp; D alternates between two block buffers
// (X32 and Yalt for float, Yalt and HX for double and double-float).
template <typename T>
cs_status cheb_ritz_core(cs_ctx* c, int n_s, double* X, long long ld, const double* HX,
                         long long ldh, const double* theta, int degree, double a, double b,
                         double a0, char* work, cudaStream_t st, bool tc = false) {
  const HostTables& H = c->host;
  const cs_precision pl = std::is_same<T, float>::value ? (tc ? CS_MIXED_BF16 : CS_FP32) : CS_FP64;
  const Layout lay = layout(c, n_s, pl);
  T* R = reinterpret_cast<T*>(work + lay.tmp);
  T* Da = std::is_same<T, float>::value ? reinterpret_cast<T*>(work + lay.X32)
                                        : reinterpret_cast<T*>(work + lay.Yalt);
  T* Db = std::is_same<T, float>::value ? reinterpret_cast<T*>(work + lay.Yalt)
                                        : reinterpret_cast<T*>(work + lay.HX);
  double* wd = reinterpret_cast<double*>(work + lay.chw);
  T* wt = reinterpret_cast<T*>(wd + (size_t)(kMaxRitzDegree + 1) * n_s);
  const double cc = 0.5 * (a + b), e = 0.5 * (b - a);
  const double s1 = e / (a0 - cc);
  CS_LAUNCH(c, 1, launch_cheb_weights<T>(theta, n_s, degree, cc, e, s1, wd, wt, st));
  CS_LAUNCH(c, 1, launch_ritz_residual<T>(X, ld, HX, ldh, theta, H.d, n_s, s1 / e, R, Da, st));
  T* cur = Da;
  T* prev = Db;
  double sig = s1;
  for (int i = 1; i < degree; ++i) {
    const double sn = 1.0 / (2.0 / s1 - sig);
    // D_{i+1} = (2 sn/e)[(H - c) D_i + s_i(Theta) R] - sig sn D_{i-1}   (D_0 = 0)
    cs_status r = hx_core<T>(c, n_s, cur, H.d, prev, H.d, EP_CHEB, 2.0 * sn / e, sig * sn, cc,
                             i == 1 ? nullptr : prev, work, st, tc, R, wt + (size_t)i * n_s);
    if (r != CS_OK) return r;
    std::swap(prev, cur);
    sig = sn;
  }
  CS_LAUNCH(c, 1, launch_ritz_combine<T>(X, ld, cur, H.d, n_s, wd + (size_t)degree * n_s, st));
  return CS_OK;
}

cs_status cheb_ritz_dispatch(cs_ctx* c, int n_s, double* X, long long ld, const double* HX,
                             long long ldh, const double* theta, int degree, double a, double b,
                             double a0, cs_precision prec, char* work, cudaStream_t st) {
  switch (prec) {
    case CS_FP64:
      return cheb_ritz_core<double>(c, n_s, X, ld, HX, ldh, theta, degree, a, b, a0, work, st);
    case CS_DF64:
      return cheb_ritz_core<df64>(c, n_s, X, ld, HX, ldh, theta, degree, a, b, a0, work, st);
    case CS_FP32:
    case CS_MIXED_BF16:
      return cheb_ritz_core<float>(c, n_s, X, ld, HX, ldh, theta, degree, a, b, a0, work, st,
                                   prec == CS_MIXED_BF16);
    default:
      return fail(c, CS_ERR_ARG, "unknown precision");
  }
}

// Gram matrix and block rotation of the ChFSI iteration in the context's dense precision
// (oz: the slice-product workspace, layout slot `oz`)
cudaError_t dense_gram(const cs_ctx* c, const double* A, long long lda, const double* B,
                       long long ldb, long long d, int na, int nb, double* C, int ldc,
                       double* part, cudaStream_t st, void* oz) {
  if (c->dense_prec == CS_FP64_SLICED)
    return launch_oz_gram(A, lda, B, ldb, d, na, nb, C, ldc, oz, c->dev_err, st);
  return c->dense_prec == CS_DF64
             ? launch_gram_df(A, lda, B, ldb, d, na, nb, C, ldc, part, st)
             : launch_gram<double>(A, lda, B, ldb, d, na, nb, C, ldc, part, st);
}
cudaError_t dense_rotate(const cs_ctx* c, const double* A, long long lda, const double* Q, int ldq,
                         long long d, int k, int n, double* C, long long ldc, cudaStream_t st,
                         void* oz, bool upper = false) {
  if (c->dense_prec == CS_FP64_SLICED)
    return launch_oz_rotate(A, lda, Q, ldq, d, k, n, C, ldc, oz, c->dev_err, st, upper);
  return c->dense_prec == CS_DF64
             ? launch_gemm_nn_df(A, lda, Q, ldq, d, k, n, 1.0, 0.0, C, ldc, st)
             : launch_gemm_nn<double>(A, lda, Q, ldq, d, k, n, 1.0, 0.0, C, ldc, st);
}

cs_status cholqr_core(cs_ctx* c, int n_s, double* X, long long ld, char* work, cudaStream_t st,
                      int* status_dev) {
  const HostTables& H = c->host;
  const Layout lay = layout(c, n_s, CS_FP64);
  double* tmp = reinterpret_cast<double*>(work + lay.tmp);
  double* part = reinterpret_cast<double*>(work + lay.part);
  double* M = reinterpret_cast<double*>(work + lay.small);
  double* U = M + (size_t)n_s * n_s;
  double* w = U + (size_t)n_s * n_s;
  void* oz = work + lay.oz;
  for (int pass = 0; pass < 2; ++pass) {
    CS_LAUNCH(c, 2, dense_gram(c, X, ld, X, ld, H.d, n_s, n_s, M, n_s, part, st, oz));
    CS_LAUNCH(c, 1, launch_cholqr_factor(M, n_s, U, w, status_dev + pass, st));
    // U = R^-1 is upper triangular with its lower part stored as zeros
    CS_LAUNCH(c, 1, dense_rotate(c, X, ld, U, n_s, H.d, n_s, n_s, tmp, H.d, st, oz, true));
    CS_LAUNCH(c, 1, launch_copy_block<double>(tmp, H.d, X, ld, H.d, n_s, st));
  }
  return CS_OK;
}

cs_status read_status(cs_ctx* c, const int* dev, int n, int* host, cudaStream_t st) {
  CS_CHECK_CUDA(c, cudaMemcpyAsync(host, dev, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
  return CS_OK;
}

cs_status rr_core(cs_ctx* c, int n_s, double* X, long long ld, double* theta, double* resid,
                  double* HX_out, char* work, cudaStream_t st, int* status_dev,
                  long long ldho = 0) {
  if (ldho == 0) ldho = ld;
  const HostTables& H = c->host;
  const Layout lay = layout(c, n_s, CS_FP64);
  double* HX = reinterpret_cast<double*>(work + lay.HX);
  double* tmp = reinterpret_cast<double*>(work + lay.tmp);
  double* part = reinterpret_cast<double*>(work + lay.part);
  double* Hs = reinterpret_cast<double*>(work + lay.small);
  double* Q = Hs + (size_t)n_s * n_s;
  double* jw = Q + (size_t)n_s * n_s;
  cs_status r;
  if (c->rr_prec == CS_FP64) {
    r = hx_core<double>(c, n_s, X, ld, HX, H.d, EP_APPLY, 0, 0, 0, nullptr, work, st);
  } else if (c->rr_prec == CS_DF64) {
    // H X in double-float: block split into tmp, product into HX, widened in place
    df64* Xd = reinterpret_cast<df64*>(work + lay.tmp);
    df64* Yd = reinterpret_cast<df64*>(work + lay.HX);
    r = hx_df64_from_fp64(c, n_s, X, ld, HX, H.d, Xd, Yd, work, st);
  } else {
    // H X in the reduced precision (FP32 block in X32, result in tmp), then back to FP64;
    // the projection, eigensolve, rotations and residual norms below stay FP64
    const Layout lr = layout(c, n_s, c->rr_prec);
    float* X32 = reinterpret_cast<float*>(work + lr.X32);
    float* HX32 = reinterpret_cast<float*>(work + lay.tmp);
    CS_LAUNCH(c, 1, launch_convert_f64_to_f32(X, ld, X32, H.d, H.d, n_s, st));
    r = hx_core<float>(c, n_s, X32, H.d, HX32, H.d, EP_APPLY, 0, 0, 0, nullptr, work, st,
                       c->rr_prec == CS_MIXED_BF16);
    if (r != CS_OK) return r;
    CS_LAUNCH(c, 1, launch_convert_f32_to_f64(HX32, H.d, HX, H.d, H.d, n_s, st));
  }
  if (r != CS_OK) return r;
  void* oz = work + lay.oz;
  CS_LAUNCH(c, 2, dense_gram(c, X, ld, HX, H.d, H.d, n_s, n_s, Hs, n_s, part, st, oz));
  // with slice-product dense steps the eigensolver's refinement products may use them too
  // (the workspace slot holds at least the d x n_s products' split operands)
  const bool sl = c->dense_prec == CS_FP64_SLICED;
  const size_t ozb = sl ? std::max(oz_gram_work_bytes(H.d, n_s, n_s, false),
                                   oz_rotate_work_bytes(H.d, n_s, n_s))
                        : 0;
  CS_LAUNCH(c, 1, launch_sym_eig(Hs, n_s, theta, Q, jw, status_dev, st, sl ? oz : nullptr, ozb,
                                 c->dev_err));
  CS_LAUNCH(c, 1, dense_rotate(c, X, ld, Q, n_s, H.d, n_s, n_s, tmp, H.d, st, oz));
  CS_LAUNCH(c, 1, launch_copy_block<double>(tmp, H.d, X, ld, H.d, n_s, st));
  // H X Q straight into HX_out when the caller keeps it, else into tmp
  double* HXq = HX_out ? HX_out : tmp;
  const long long ldq = HX_out ? ldho : H.d;
  CS_LAUNCH(c, 1, dense_rotate(c, HX, H.d, Q, n_s, H.d, n_s, n_s, HXq, ldq, st, oz));
  CS_LAUNCH(c, 1, launch_residuals(X, ld, HXq, ldq, H.d, n_s, theta, resid, st));
  return CS_OK;
}

cs_status hx_df64_from_fp64(cs_ctx* c, int n_s, const double* X, long long ld, double* HX,
                            long long ldh, df64* Xd, df64* Yd, char* work, cudaStream_t st) {
  const HostTables& H = c->host;
  const Layout lay = layout(c, n_s, CS_FP64);
  const df64* kb = nullptr;
  if (c->n_p > 0) {
    if (c->dense_prec != CS_FP64_SLICED)
      return fail(c, CS_ERR_STATE,
                  "CS_DF64 applies projectors only with CS_FP64_SLICED dense products");
    double* Wkb = reinterpret_cast<double*>(work + lay.Wkb);
    double* kbZ = reinterpret_cast<double*>(work + lay.kbZ);
    void* oz = work + lay.oz;
    CS_LAUNCH_CLS(c, prof_cls<df64>(4), 4,
                  launch_oz_gram(c->d64.pcoef, H.d, X, ld, H.d, c->n_p, n_s, Wkb, c->n_p, oz,
                                 c->dev_err, st));
    CS_LAUNCH_CLS(c, prof_cls<df64>(4), 1,
                  launch_scale_rows<double>(Wkb, c->n_p, n_s, c->n_p, c->d64.h, st));
    CS_LAUNCH_CLS(c, prof_cls<df64>(4), 4,
                  launch_oz_rotate(c->d64.pcoef, H.d, Wkb, c->n_p, H.d, c->n_p, n_s, kbZ, H.d, oz,
                                   c->dev_err, st));
    CS_LAUNCH(c, 1, launch_to_df64(kbZ, H.d, reinterpret_cast<df64*>(kbZ), H.d, H.d, n_s, st));
    kb = reinterpret_cast<const df64*>(kbZ);
  }
  CS_LAUNCH(c, 1, launch_to_df64(X, ld, Xd, H.d, H.d, n_s, st));
  cs_status r = hx_core<df64>(c, n_s, Xd, H.d, Yd, H.d, EP_APPLY, 0, 0, 0, nullptr, work, st,
                              false, nullptr, nullptr, kb);
  if (r != CS_OK) return r;
  CS_LAUNCH(c, 1, launch_from_df64(Yd, H.d, HX, ldh, H.d, n_s, st));
  return CS_OK;
}

// reads and clears the device error word (synchronising)
cs_status check_dev_err(cs_ctx* c, cudaStream_t st) {
  if (!c->dev_err) return CS_OK;
  int code = 0;
  CS_CHECK_CUDA(c, cudaMemcpyAsync(&code, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
  if (code != 0) {
    CS_CHECK_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), st));
    return fail(c, CS_ERR_TIMEOUT, "a bounded device wait expired (code " + std::to_string(code) + ")");
  }
  return CS_OK;
}

// filter (precision prec) -> Cholesky-QR (FP64) -> Rayleigh-Ritz (FP64); synchronising.
// With ritz_HX the filter takes the residual form: X are Ritz vectors, ritz_HX their H X and
// theta their Ritz values (all on entry). HX_out (may equal ritz_HX) receives H X of the new
// Ritz vectors.
cs_status chfsi_step_core(cs_ctx* c, int n_s, double* X, long long ld, int degree, double a,
                          double b, double a0, cs_precision prec, double* theta, double* resid,
                          char* wk, cudaStream_t st, const double* ritz_HX = nullptr,
                          double* HX_out = nullptr, long long ldh = 0) {
  if (ldh == 0) ldh = ld;
  const HostTables& H = c->host;
  const Layout lay = layout(c, n_s, prec);
  int* status = reinterpret_cast<int*>(wk + lay.status);
  cs_status s;
  if (ritz_HX) {
    s = cheb_ritz_dispatch(c, n_s, X, ld, ritz_HX, ldh, theta, degree, a, b, a0, prec, wk, st);
  } else if (prec == CS_FP64) {
    s = cheb_core<double>(c, n_s, X, ld, degree, a, b, a0, wk, st);
  } else if (prec == CS_DF64) {
    df64* Xd = reinterpret_cast<df64*>(wk + lay.tmp);
    CS_LAUNCH(c, 1, launch_to_df64(X, ld, Xd, H.d, H.d, n_s, st));
    s = cheb_core<df64>(c, n_s, Xd, H.d, degree, a, b, a0, wk, st);
    if (s == CS_OK) CS_LAUNCH(c, 1, launch_from_df64(Xd, H.d, X, ld, H.d, n_s, st));
  } else {
    float* X32 = reinterpret_cast<float*>(wk + lay.X32);
    CS_LAUNCH(c, 1, launch_convert_f64_to_f32(X, ld, X32, H.d, H.d, n_s, st));
    s = cheb_core<float>(c, n_s, X32, H.d, degree, a, b, a0, wk, st, prec == CS_MIXED_BF16);
    if (s == CS_OK) CS_LAUNCH(c, 1, launch_convert_f32_to_f64(X32, H.d, X, ld, H.d, n_s, st));
  }
  if (s != CS_OK) return s;
  if ((s = cholqr_core(c, n_s, X, ld, wk, st, status)) != CS_OK) return s;
  if ((s = rr_core(c, n_s, X, ld, theta, resid, HX_out, wk, st, status + 4, ldh)) != CS_OK)
    return s;
  int hs[5];
  if ((s = read_status(c, status, 5, hs, st)) != CS_OK) return s;
  if ((s = check_dev_err(c, st)) != CS_OK) return s;
  if (hs[0] != 0 || hs[1] != 0) return fail(c, CS_ERR_CHOLESKY, "Cholesky breakdown in ChFSI");
  if (hs[4] < 0) return fail(c, CS_ERR_NOT_CONVERGED, "Jacobi eigensolver did not converge");
  return CS_OK;
}

cs_status check_block(cs_ctx* c, int n_s, const void* X, long long ld) {
  if (n_s < 1) return fail(c, CS_ERR_ARG, "n_s must be >= 1");
  if (ld < c->host.d) return fail(c, CS_ERR_ARG, "ld must be >= d");
  if (!X) return fail(c, CS_ERR_ARG, "block pointer is NULL");
  return CS_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

cs_status cs_basis_init(double R, int lmax, int nmax, const cs_quadrature* q, int cuda_device,
                        cs_ctx** out) {
  if (!out || !q) {
    g_init_error = "NULL argument";
    return CS_ERR_ARG;
  }
  *out = nullptr;
  cs_ctx* c = new (std::nothrow) cs_ctx();
  if (!c) {
    g_init_error = "host allocation failed";
    return CS_ERR_ALLOC;
  }
  std::string msg = build_host_tables(R, lmax, nmax, *q, c->host);
  if (!msg.empty()) {
    g_init_error = msg;
    delete c;
    return CS_ERR_ARG;
  }
  c->Q4 = c->host.n_phi / 4;
  if (cuda_device >= 0) {
    if (cudaSetDevice(cuda_device) != cudaSuccess) {
      g_init_error = "cudaSetDevice failed";
      delete c;
      return CS_ERR_CUDA;
    }
    c->device = cuda_device;
    c->has_device = true;
    if (pick_states_per_cta<double>(c->host.L, c->host.n_phi, c->Q4) == 0) {
      g_init_error = "lmax too large for the angular kernel's shared-memory tile";
      cs_basis_free(c);
      return CS_ERR_ARG;
    }
    cs_status st = upload_tables<double>(c);
    if (st == CS_OK) st = upload_tables<float>(c);
    if (st == CS_OK) st = upload_tables<df64>(c);
    if (st == CS_OK) {
      for (int mode = 0; mode < 2 && st == CS_OK; ++mode) {
        std::vector<uint16_t> tab;
        int mt = 0, kp = 0;
        build_tc_tables(c->host, mode, tab, mt, kp);
        void** dst = mode == 0 ? &c->tc_synth : &c->tc_anal;
        if (cudaMalloc(dst, tab.size() * 2) != cudaSuccess ||
            cudaMemcpy(*dst, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
          st = CS_ERR_ALLOC;
        if (mode == 0) {
          c->tc_rows_synth = mt;
          c->tc_kpad_synth = kp;
        } else {
          c->tc_rows_anal = mt;
          c->tc_kpad_anal = kp;
        }
      }
      if (st == CS_OK && angular_tc_eligible(c->host.L, c->host.n_theta, c->host.n_phi)) {
        std::vector<uint16_t> tab;
        build_tc_phi_table(c->host.L, c->host.n_phi, tab);
        if (cudaMalloc(&c->tc_phi, tab.size() * 2) != cudaSuccess ||
            cudaMemcpy(c->tc_phi, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice) !=
                cudaSuccess)
          st = CS_ERR_ALLOC;
      }
      if (st == CS_OK && angular_wide_eligible(c->host.L, c->host.n_theta, c->host.n_phi)) {
        std::vector<uint16_t> tab;
        build_wide_tables(c->host, tab);
        if (cudaMalloc(&c->wide_tab, tab.size() * 2) != cudaSuccess ||
            cudaMemcpy(c->wide_tab, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice) !=
                cudaSuccess)
          st = CS_ERR_ALLOC;
      }
      if (st == CS_OK && (cudaMalloc((void**)&c->dev_err, sizeof(int)) != cudaSuccess ||
                          cudaMemset(c->dev_err, 0, sizeof(int)) != cudaSuccess))
        st = CS_ERR_ALLOC;
    }
    if (st == CS_OK) {
      size_t nr = c->host.w_r.size();
      if (cudaMalloc((void**)&c->w_r_dev, nr * sizeof(double)) != cudaSuccess ||
          cudaMemcpy(c->w_r_dev, c->host.w_r.data(), nr * sizeof(double),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        st = CS_ERR_ALLOC;
    }
    if (st == CS_OK) {
      // Hartree tables: k_ln = z_ln / R ([l][n]), then r_k / R ([k])
      const HostTables& H = c->host;
      std::vector<double> tab((size_t)H.L * H.N + H.n_r);
      for (size_t i = 0; i < (size_t)H.L * H.N; ++i) tab[i] = H.z[i] / H.R;
      for (int k = 0; k < H.n_r; ++k) tab[(size_t)H.L * H.N + k] = H.r[k] / H.R;
      if (cudaMalloc((void**)&c->hartree_tab, tab.size() * sizeof(double)) != cudaSuccess ||
          cudaMemcpy(c->hartree_tab, tab.data(), tab.size() * sizeof(double),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        st = CS_ERR_ALLOC;
    }
    if (st == CS_OK) {
      // grid coordinates: r_k, cos(theta_j), phi_q
      const HostTables& H = c->host;
      std::vector<double> g;
      g.insert(g.end(), H.r.begin(), H.r.end());
      g.insert(g.end(), H.t.begin(), H.t.end());
      g.insert(g.end(), H.phi.begin(), H.phi.end());
      if (cudaMalloc((void**)&c->grid_tab, g.size() * sizeof(double)) != cudaSuccess ||
          cudaMemcpy(c->grid_tab, g.data(), g.size() * sizeof(double),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        st = CS_ERR_ALLOC;
    }
    if (st != CS_OK) {
      g_init_error = c->err;
      cs_basis_free(c);
      return st;
    }
  }
  *out = c;
  return CS_OK;
}

cs_status cs_basis_free(cs_ctx* c) {
  if (!c) return CS_OK;
  if (c->has_device) {
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_tables(c->d64);
    free_tables(c->d32);
    free_tables(c->ddf);
    for (auto& r : c->prof_recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->w_r_dev) cudaFree(c->w_r_dev);
    if (c->hartree_tab) cudaFree(c->hartree_tab);
    if (c->grid_tab) cudaFree(c->grid_tab);
    if (c->tc_synth) cudaFree(c->tc_synth);
    if (c->tc_anal) cudaFree(c->tc_anal);
    if (c->tc_phi) cudaFree(c->tc_phi);
    if (c->wide_tab) cudaFree(c->wide_tab);
    if (c->kb_tabA) cudaFree(c->kb_tabA);
    if (c->kb_tabB) cudaFree(c->kb_tabB);
    if (c->dev_err) cudaFree(c->dev_err);
  }
  delete c;
  return CS_OK;
}

cs_status cs_basis_dims(const cs_ctx* c, long long* d, int* n_r, int* n_theta, int* n_phi) {
  if (!c) return CS_ERR_ARG;
  if (d) *d = c->host.d;
  if (n_r) *n_r = c->host.n_r;
  if (n_theta) *n_theta = c->host.n_theta;
  if (n_phi) *n_phi = c->host.n_phi;
  return CS_OK;
}

cs_status cs_grid(const cs_ctx* c, double* r, double* w_r, double* t, double* w_t, double* phi) {
  if (!c) return CS_ERR_ARG;
  const HostTables& H = c->host;
  if (r) std::memcpy(r, H.r.data(), H.r.size() * 8);
  if (w_r) std::memcpy(w_r, H.w_r.data(), H.w_r.size() * 8);
  if (t) std::memcpy(t, H.t.data(), H.t.size() * 8);
  if (w_t) std::memcpy(w_t, H.w_t.data(), H.w_t.size() * 8);
  if (phi) std::memcpy(phi, H.phi.data(), H.phi.size() * 8);
  return CS_OK;
}

cs_status cs_kinetic(const cs_ctx* c, double* half_lambda) {
  if (!c || !half_lambda) return CS_ERR_ARG;
  std::memcpy(half_lambda, c->host.half_lambda.data(), c->host.half_lambda.size() * 8);
  return CS_OK;
}

cs_status cs_bessel_zeros(const cs_ctx* c, double* z) {
  if (!c || !z) return CS_ERR_ARG;
  std::memcpy(z, c->host.z.data(), c->host.z.size() * 8);
  return CS_OK;
}

cs_status cs_set_potential(cs_ctx* c, const double* v_grid, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if (!v_grid) return fail(c, CS_ERR_ARG, "v_grid is NULL");
  const HostTables& H = c->host;
  cudaStream_t st = (cudaStream_t)stream;
  CS_LAUNCH(c, 1, launch_weighted_potential(v_grid, c->d64.wkj, H.n_r * H.n_theta, H.n_phi,
                                            c->d64.wv, c->d32.wv, c->ddf.wv, st));
  c->has_potential = true;
  return CS_OK;
}

cs_status cs_set_projectors(cs_ctx* c, int n_p, const double* p_coef, const double* h,
                            cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if (n_p < 0 || (n_p > 0 && (!p_coef || !h))) return fail(c, CS_ERR_ARG, "bad projector arguments");
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
  for (void** p : {(void**)&c->d64.pcoef, (void**)&c->d64.h, (void**)&c->d32.pcoef,
                   (void**)&c->d32.h, &c->kb_tabA, &c->kb_tabB}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  c->n_p = 0;
  if (n_p == 0) return CS_OK;
  const size_t d = (size_t)c->host.d;
  const KbTcShape ks = kb_tc_shape(c->host.d, n_p, 1);
  if (cudaMalloc((void**)&c->d64.pcoef, d * n_p * 8) != cudaSuccess ||
      cudaMalloc((void**)&c->d32.pcoef, d * n_p * 4) != cudaSuccess ||
      cudaMalloc(&c->kb_tabA, ks.tabA_bytes) != cudaSuccess ||
      cudaMalloc(&c->kb_tabB, ks.tabB_bytes) != cudaSuccess)
    return fail(c, CS_ERR_ALLOC, "cudaMalloc of projector tables failed");
  cs_status r;
  std::vector<double> hv(h, h + n_p);
  if ((r = upload<double>(c, &c->d64.h, hv)) != CS_OK) return r;
  if ((r = upload<float>(c, &c->d32.h, hv)) != CS_OK) return r;
  CS_CHECK_CUDA(c, cudaMemcpyAsync(c->d64.pcoef, p_coef, d * n_p * 8, cudaMemcpyDeviceToDevice, st));
  CS_LAUNCH(c, 1, launch_convert_f64_to_f32(c->d64.pcoef, (long long)d, c->d32.pcoef,
                                            (long long)d, (long long)d, n_p, st));
  CS_LAUNCH(c, 2, build_kb_tc_tables(c->d64.pcoef, (long long)d, n_p, c->kb_tabA, c->kb_tabB, st));
  CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
  c->n_p = n_p;
  return CS_OK;
}

cs_status cs_set_rr_precision(cs_ctx* c, cs_precision prec) {
  if (!c) return CS_ERR_ARG;
  if (prec != CS_FP64 && prec != CS_FP32 && prec != CS_MIXED_BF16 && prec != CS_DF64)
    return fail(c, CS_ERR_ARG, "unknown precision");
  c->rr_prec = prec;
  return CS_OK;
}

cs_status cs_set_dense_precision(cs_ctx* c, cs_precision prec) {
  if (!c) return CS_ERR_ARG;
  if (prec != CS_FP64 && prec != CS_DF64 && prec != CS_FP64_SLICED)
    return fail(c, CS_ERR_ARG, "dense precision must be CS_FP64, CS_DF64 or CS_FP64_SLICED");
  c->dense_prec = prec;
  return CS_OK;
}

cs_status cs_dense_gram(cs_ctx* c, int na, int nb, const double* A, long long lda,
                        const double* B, long long ldb, double* C, long long ldc, void* work,
                        cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  const long long d = c->host.d;
  if (na < 1 || nb < 1 || !A || !B || !C || !work || lda < d || ldb < d || ldc < na ||
      ldc > 0x7fffffff)
    return fail(c, CS_ERR_ARG, "bad Gram arguments");
  const int n = std::max(na, nb);
  const Layout lay = layout(c, n, CS_FP64);
  char* wk = (char*)work;
  cudaStream_t st = (cudaStream_t)stream;
  CS_LAUNCH(c, 2, dense_gram(c, A, lda, B, ldb, d, na, nb, C, (int)ldc,
                             reinterpret_cast<double*>(wk + lay.part), st, wk + lay.oz));
  return CS_OK;
}

cs_status cs_dense_rotate(cs_ctx* c, int k, int n, const double* A, long long lda,
                          const double* Q, long long ldq, double* C, long long ldc, void* work,
                          cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  const long long d = c->host.d;
  if (k < 1 || n < 1 || !A || !Q || !C || !work || lda < d || ldc < d || ldq < k ||
      ldq > 0x7fffffff || A == C)
    return fail(c, CS_ERR_ARG, "bad rotation arguments");
  const Layout lay = layout(c, std::max(k, n), CS_FP64);
  cudaStream_t st = (cudaStream_t)stream;
  CS_LAUNCH(c, 1, dense_rotate(c, A, lda, Q, (int)ldq, d, k, n, C, ldc, st, (char*)work + lay.oz));
  return CS_OK;
}

cs_status cs_workspace_bytes(const cs_ctx* c, int n_s, cs_precision prec, size_t* bytes) {
  if (!c || !bytes || n_s < 1) return CS_ERR_ARG;
  *bytes = layout(c, n_s, prec).total;
  return CS_OK;
}

cs_status cs_forward_transform(cs_ctx* c, int n, const double* g, double* coef, long long ld,
                               void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n, coef, ld)) != CS_OK) return s;
  if (!g || !work) return fail(c, CS_ERR_ARG, "NULL grid or workspace");
  const HostTables& H = c->host;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout lay = layout(c, n, CS_FP64);
  double* G = reinterpret_cast<double*>((char*)work + lay.G);
  AngArgs<double> a{H.L, H.n_r, H.n_theta, H.n_phi, c->Q4, n, c->d64.theta, c->d64.trig,
                    c->d64.wv, c->d64.wkj};
  CS_LAUNCH(c, 1, launch_angular<double>(a, ANG_ANAL, G, nullptr, g, st));
  Epilogue<double> ep;
  ep.mode = EP_PLAIN;
  ep.out = coef;
  ep.ld_out = ld;
  CS_LAUNCH(c, 1, launch_radial_anal<double>(G, c->d64.rad, H.L, H.N, H.n_r, n, ep, st));
  return CS_OK;
}

cs_status cs_inverse_transform(cs_ctx* c, int n, const double* coef, long long ld, double* f,
                               void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n, coef, ld)) != CS_OK) return s;
  if (!f || !work) return fail(c, CS_ERR_ARG, "NULL grid or workspace");
  const HostTables& H = c->host;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout lay = layout(c, n, CS_FP64);
  double* G = reinterpret_cast<double*>((char*)work + lay.G);
  CS_LAUNCH(c, 1, launch_radial_synth<double>(coef, ld, G, c->d64.rad, H.L, H.N, H.n_r, n, st));
  AngArgs<double> a{H.L, H.n_r, H.n_theta, H.n_phi, c->Q4, n, c->d64.theta, c->d64.trig,
                    c->d64.wv, c->d64.wkj};
  CS_LAUNCH(c, 1, launch_angular<double>(a, ANG_SYNTH, G, f, nullptr, st));
  return CS_OK;
}

cs_status cs_apply_H(cs_ctx* c, int n_s, const void* X, void* HX, long long ld,
                     cs_precision prec, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!HX || !work) return fail(c, CS_ERR_ARG, "NULL output or workspace");
  if (X == HX) return fail(c, CS_ERR_ARG, "X and HX must not overlap");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CS_FP64)
    return hx_core<double>(c, n_s, (const double*)X, ld, (double*)HX, ld, EP_APPLY, 0, 0, 0,
                           nullptr, (char*)work, st);
  if (prec == CS_FP32 || prec == CS_MIXED_BF16)
    return hx_core<float>(c, n_s, (const float*)X, ld, (float*)HX, ld, EP_APPLY, 0, 0, 0,
                          nullptr, (char*)work, st, prec == CS_MIXED_BF16);
  if (prec == CS_DF64) {
    const Layout lay = layout(c, n_s, CS_DF64);
    df64* Xd = reinterpret_cast<df64*>((char*)work + lay.tmp);
    df64* Yd = reinterpret_cast<df64*>((char*)work + lay.HX);
    return hx_df64_from_fp64(c, n_s, (const double*)X, ld, (double*)HX, ld, Xd, Yd,
                             (char*)work, st);
  }
  return fail(c, CS_ERR_ARG, "unknown precision");
}

cs_status cs_cheb_filter(cs_ctx* c, int n_s, void* X, long long ld, int degree, double a,
                         double b, double a0, cs_precision prec, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!work) return fail(c, CS_ERR_ARG, "NULL workspace");
  if (degree < 1) return fail(c, CS_ERR_ARG, "degree must be >= 1");
  if (!(a < b) || !(a0 < a)) return fail(c, CS_ERR_ARG, "need a0 < a < b");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CS_FP64) return cheb_core<double>(c, n_s, (double*)X, ld, degree, a, b, a0, (char*)work, st);
  if (prec == CS_FP32 || prec == CS_MIXED_BF16)
    return cheb_core<float>(c, n_s, (float*)X, ld, degree, a, b, a0, (char*)work, st,
                            prec == CS_MIXED_BF16);
  if (prec == CS_DF64) {
    const HostTables& H = c->host;
    df64* Xd = reinterpret_cast<df64*>((char*)work + layout(c, n_s, CS_DF64).tmp);
    CS_LAUNCH(c, 1, launch_to_df64((const double*)X, ld, Xd, H.d, H.d, n_s, st));
    cs_status r = cheb_core<df64>(c, n_s, Xd, H.d, degree, a, b, a0, (char*)work, st);
    if (r != CS_OK) return r;
    CS_LAUNCH(c, 1, launch_from_df64(Xd, H.d, (double*)X, ld, H.d, n_s, st));
    return CS_OK;
  }
  return fail(c, CS_ERR_ARG, "unknown precision");
}

cs_status cs_cholqr(cs_ctx* c, int n_s, double* X, long long ld, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!work) return fail(c, CS_ERR_ARG, "NULL workspace");
  if (n_s > 1024) return fail(c, CS_ERR_ARG, "n_s > 1024 not supported");
  cudaStream_t st = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>((char*)work + layout(c, n_s, CS_FP64).status);
  if ((s = cholqr_core(c, n_s, X, ld, (char*)work, st, status)) != CS_OK) return s;
  int hs[2];
  if ((s = read_status(c, status, 2, hs, st)) != CS_OK) return s;
  if (hs[0] != 0 || hs[1] != 0)
    return fail(c, CS_ERR_CHOLESKY, "Cholesky breakdown at pivot " + std::to_string(hs[0] ? hs[0] - 1 : hs[1] - 1));
  return CS_OK;
}

cs_status cs_rayleigh_ritz(cs_ctx* c, int n_s, double* X, long long ld, double* theta,
                           double* resid, double* HX_out, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!theta || !resid || !work) return fail(c, CS_ERR_ARG, "NULL theta, resid or workspace");
  if (n_s > 1024) return fail(c, CS_ERR_ARG, "n_s > 1024 not supported");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  cudaStream_t st = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>((char*)work + layout(c, n_s, CS_FP64).status);
  if ((s = rr_core(c, n_s, X, ld, theta, resid, HX_out, (char*)work, st, status + 4)) != CS_OK)
    return s;
  int hs;
  if ((s = read_status(c, status + 4, 1, &hs, st)) != CS_OK) return s;
  if (hs < 0) return fail(c, CS_ERR_NOT_CONVERGED, "Jacobi eigensolver did not converge");
  return CS_OK;
}

cs_status cs_lanczos_bound(cs_ctx* c, int k, const double* v0, double* b, double* theta_min,
                           void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if (k < 1 || k > kMaxLanczos || !v0 || !b || !theta_min || !work)
    return fail(c, CS_ERR_ARG, "bad Lanczos arguments (1 <= k <= 64)");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  const HostTables& H = c->host;
  const long long d = H.d;
  cudaStream_t st = (cudaStream_t)stream;
  char* wk = (char*)work;
  const Layout lay = layout(c, 1, CS_FP64);
  double* V = reinterpret_cast<double*>(wk + lay.lanV);  // d x (k+1), then w
  double* w = V + (size_t)d * (kMaxLanczos + 1);
  double* part = reinterpret_cast<double*>(wk + lay.part);
  double* sm = reinterpret_cast<double*>(wk + lay.small);
  double* alpha = sm;                  // [k]
  double* beta2 = alpha + kMaxLanczos; // [k]
  double* dots = beta2 + kMaxLanczos;  // [k+1]
  double* nrm = dots + kMaxLanczos + 2;
  double* T = nrm + 4;                 // k x k
  double* Q = T + kMaxLanczos * kMaxLanczos;
  double* th = Q + kMaxLanczos * kMaxLanczos;
  double* jw = th + kMaxLanczos;
  int* status = reinterpret_cast<int*>(wk + lay.status);
  CS_LAUNCH(c, 2, launch_gram(v0, d, v0, d, d, 1, 1, nrm, 1, part, st));
  CS_LAUNCH(c, 1, launch_scale_inv_sqrt(v0, V, d, nrm, st));
  for (int i = 0; i < k; ++i) {
    double* vi = V + (size_t)i * d;
    s = hx_core<double>(c, 1, vi, d, w, d, EP_APPLY, 0, 0, 0, nullptr, wk, st);
    if (s != CS_OK) return s;
    // alpha_i = v_i . w ; full re-orthogonalisation against v_0 .. v_i (twice)
    CS_LAUNCH(c, 2, launch_gram(V, d, w, d, d, i + 1, 1, dots, i + 1, part, st));
    CS_CHECK_CUDA(c, cudaMemcpyAsync(alpha + i, dots + i, 8, cudaMemcpyDeviceToDevice, st));
    CS_LAUNCH(c, 1, launch_gemm_nn(V, d, dots, i + 1, d, i + 1, 1, -1.0, 1.0, w, d, st));
    CS_LAUNCH(c, 2, launch_gram(V, d, w, d, d, i + 1, 1, dots, i + 1, part, st));
    CS_LAUNCH(c, 1, launch_gemm_nn(V, d, dots, i + 1, d, i + 1, 1, -1.0, 1.0, w, d, st));
    CS_LAUNCH(c, 2, launch_gram(w, d, w, d, d, 1, 1, beta2 + i, 1, part, st));
    CS_LAUNCH(c, 1, launch_scale_inv_sqrt(w, V + (size_t)(i + 1) * d, d, beta2 + i, st));
  }
  CS_LAUNCH(c, 1, launch_build_tridiag(alpha, beta2, k, T, st));
  CS_LAUNCH(c, 1, launch_sym_eig(T, k, th, Q, jw, status + 8, st));
  std::vector<double> hth(k), hb2(k);
  CS_CHECK_CUDA(c, cudaMemcpyAsync(hth.data(), th, k * 8, cudaMemcpyDeviceToHost, st));
  CS_CHECK_CUDA(c, cudaMemcpyAsync(hb2.data(), beta2, k * 8, cudaMemcpyDeviceToHost, st));
  CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
  *b = hth[k - 1] + std::sqrt(hb2[k - 1]);
  *theta_min = hth[0];
  if (!std::isfinite(*b) || !std::isfinite(*theta_min))
    return fail(c, CS_ERR_NUMERIC, "Lanczos produced a non-finite bound (breakdown?)");
  return CS_OK;
}

cs_status cs_chfsi(cs_ctx* c, int n_s, int n_want, double* X, long long ld, int degree,
                   double tol, int max_iter, cs_precision prec, const double* v0, double* theta,
                   double* resid, int* iters, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (n_want < 1 || n_want > n_s || degree < 1 || max_iter < 1 || !v0 || !theta || !resid ||
      !work)
    return fail(c, CS_ERR_ARG, "bad ChFSI arguments");
  if (prec != CS_FP64 && prec != CS_FP32 && prec != CS_MIXED_BF16 && prec != CS_DF64)
    return fail(c, CS_ERR_ARG, "unknown precision");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  const HostTables& H = c->host;
  cudaStream_t st = (cudaStream_t)stream;
  char* wk = (char*)work;
  const Layout lay = layout(c, n_s, prec);
  int* status = reinterpret_cast<int*>(wk + lay.status);
  double bnd = 0, tmin = 0;
  if ((s = cs_lanczos_bound(c, 10, v0, &bnd, &tmin, work, stream)) != CS_OK) return s;
  double a0 = tmin, a = a0 + (bnd - a0) / 10.0;
  if ((s = cs_cholqr(c, n_s, X, ld, work, stream)) != CS_OK) return s;
  std::vector<double> hth(n_s), hres(n_s);
  // FP32 and mixed filters run in residual form once Ritz vectors exist: their H.X rounding
  // then scales with the residual, so the iteration converges past the filter's precision
  const bool ritz = (prec == CS_FP32 || prec == CS_MIXED_BF16) && degree <= kMaxRitzDegree;
  double* HXr = reinterpret_cast<double*>(wk + lay.HXr);
  int it = 0;
  bool conv = false;
  for (it = 1; it <= max_iter; ++it) {
    const bool use_ritz = ritz && it > 1;
    if ((s = chfsi_step_core(c, n_s, X, ld, degree, a, bnd, a0, prec, theta, resid, wk, st,
                             use_ritz ? HXr : nullptr, ritz ? HXr : nullptr, H.d)) != CS_OK)
      return s;
    CS_CHECK_CUDA(c, cudaMemcpyAsync(hth.data(), theta, n_s * 8, cudaMemcpyDeviceToHost, st));
    CS_CHECK_CUDA(c, cudaMemcpyAsync(hres.data(), resid, n_s * 8, cudaMemcpyDeviceToHost, st));
    CS_CHECK_CUDA(c, cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int i = 0; i < n_want; ++i) worst = std::max(worst, hres[i]);
    if (!std::isfinite(worst)) return fail(c, CS_ERR_NUMERIC, "non-finite residual in ChFSI");
    if (worst <= tol) {
      conv = true;
      break;
    }
    a = hth[n_s - 1];
    a0 = hth[0];
  }
  if (iters) *iters = conv ? it : max_iter;
  if (!conv) return fail(c, CS_ERR_NOT_CONVERGED, "ChFSI reached max_iter");
  return CS_OK;
}

cs_status cs_chfsi_step(cs_ctx* c, int n_s, double* X, long long ld, int degree, double a,
                        double b, double a0, cs_precision prec, double* theta, double* resid,
                        void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (degree < 1 || !theta || !resid || !work) return fail(c, CS_ERR_ARG, "bad ChFSI step arguments");
  if (!(a < b) || !(a0 < a)) return fail(c, CS_ERR_ARG, "need a0 < a < b");
  if (n_s > 1024) return fail(c, CS_ERR_ARG, "n_s > 1024 not supported");
  if (prec != CS_FP64 && prec != CS_FP32 && prec != CS_MIXED_BF16 && prec != CS_DF64)
    return fail(c, CS_ERR_ARG, "unknown precision");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  return chfsi_step_core(c, n_s, X, ld, degree, a, b, a0, prec, theta, resid, (char*)work,
                         (cudaStream_t)stream);
}

cs_status cs_cheb_filter_ritz(cs_ctx* c, int n_s, double* X, long long ld, const double* HX,
                              long long ldh, const double* theta, int degree, double a, double b,
                              double a0, cs_precision prec, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!HX || !theta || !work) return fail(c, CS_ERR_ARG, "NULL HX, theta or workspace");
  if (ldh < c->host.d) return fail(c, CS_ERR_ARG, "ldh must be >= d");
  if (degree < 1 || degree > kMaxRitzDegree)
    return fail(c, CS_ERR_ARG, "degree must be in 1 .. 64 for the residual-form filter");
  if (!(a < b) || !(a0 < a)) return fail(c, CS_ERR_ARG, "need a0 < a < b");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  return cheb_ritz_dispatch(c, n_s, X, ld, HX, ldh, theta, degree, a, b, a0, prec, (char*)work,
                            (cudaStream_t)stream);
}

cs_status cs_chfsi_step_ritz(cs_ctx* c, int n_s, double* X, double* HX, long long ld, int degree,
                             double a, double b, double a0, cs_precision prec, double* theta,
                             double* resid, void* work, cs_stream stream) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if ((s = check_block(c, n_s, X, ld)) != CS_OK) return s;
  if (!HX || HX == X || !theta || !resid || !work)
    return fail(c, CS_ERR_ARG, "bad ChFSI step arguments");
  if (degree < 1 || degree > kMaxRitzDegree)
    return fail(c, CS_ERR_ARG, "degree must be in 1 .. 64 for the residual-form filter");
  if (!(a < b) || !(a0 < a)) return fail(c, CS_ERR_ARG, "need a0 < a < b");
  if (n_s > 1024) return fail(c, CS_ERR_ARG, "n_s > 1024 not supported");
  if (prec != CS_FP64 && prec != CS_FP32 && prec != CS_MIXED_BF16 && prec != CS_DF64)
    return fail(c, CS_ERR_ARG, "unknown precision");
  if (!c->has_potential) return fail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  return chfsi_step_core(c, n_s, X, ld, degree, a, b, a0, prec, theta, resid, (char*)work,
                         (cudaStream_t)stream, HX, HX, ld);
}

cs_status cs_device_error(cs_ctx* c, int* code) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if (!code) return fail(c, CS_ERR_ARG, "NULL code");
  CS_CHECK_CUDA(c, cudaMemcpy(code, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  CS_CHECK_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
  return CS_OK;
}

cs_status cs_profile_begin(cs_ctx* c) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  c->prof = true;
  return CS_OK;
}

cs_status cs_profile_end(cs_ctx* c, double* ms, long long* launches) {
  cs_status s = need_device(c);
  if (s != CS_OK) return s;
  if (!ms || !launches) return fail(c, CS_ERR_ARG, "NULL output");
  for (int i = 0; i < CS_PROFILE_CLASSES; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (auto& r : c->prof_recs) {
    CS_CHECK_CUDA(c, cudaEventSynchronize(r.b));
    float t = 0.f;
    CS_CHECK_CUDA(c, cudaEventElapsedTime(&t, r.a, r.b));
    if (r.cls >= 0 && r.cls < CS_PROFILE_CLASSES) {
      ms[r.cls] += t;
      launches[r.cls] += 1;
    }
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->prof_recs.clear();
  c->prof = false;
  return CS_OK;
}

const char* cs_last_error(const cs_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}

long long cs_launch_count(const cs_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
