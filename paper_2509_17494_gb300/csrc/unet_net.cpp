// Learned coarse corrector: the network's buffers and launch sequences (see
// unet_net.h; the layer arithmetic is in unet.cu).  Parameter order, layer
// order and the backward chain follow the architecture description in unet.cu:
// encoder levels 0..L-1 (two convolutions each, average pooling between
// levels), decoder levels L-2..0 (nearest doubling into the second half of a
// concatenation buffer whose first half the encoder wrote, two convolutions),
// then the 1x1 head.
#include "unet_net.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "unet.h"

namespace th {

namespace {
#define UN_CU(expr)                              \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return _e;            \
  } while (0)
}  // namespace

int UNet::check(int levels, int base) {
  if (levels < 2 || levels > 6 || base < 16 || (base & 15)) return 0;
  // the widest forward output (the bottom level) must fit one MMA (N <= 256);
  // input gradients wider than that (decoder concatenations) are split
  const int top = base << (levels - 1);
  if (top > 256 || (base << (levels - 2)) * 3 > 1024) return 0;
  return 1;
}

size_t UNet::param_count(int levels, int base) {
  size_t n = 0;
  int prev = 3;
  for (int l = 0; l < levels; ++l) {
    const int c = base << l;
    n += (size_t)c * 9 * prev + c + (size_t)c * 9 * c + c;
    prev = c;
  }
  for (int l = levels - 2; l >= 0; --l) {
    const int c = base << l, cu = base << (l + 1);
    n += (size_t)c * 9 * (c + cu) + c + (size_t)c * 9 * c + c;
  }
  return n + 2 * (size_t)base + 2;
}

template <typename T>
T* UNet::alloc(size_t n) {
  void* p = nullptr;
  if (!ok_ || cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    ok_ = false;
    return nullptr;
  }
  cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(T));
  owned_.push_back(p);
  return static_cast<T*>(p);
}

UNet::UNet(int levels, int base, int batch_max, int m, const std::vector<float>& eta, int* err)
    : L_(levels), base_(base), bmax_(batch_max), m_(m), err_(err) {
  if (!check(levels, base) || batch_max < 1 || m < 2 || (int)eta.size() != m * m) {
    ok_ = false;
    return;
  }
  const int q = 1 << (L_ - 1);
  mp_ = (m + q - 1) / q * q;
  for (int l = 0; l < L_; ++l) C_.push_back(base << l);
  // parameter layout (oracle order)
  size_t off = 0;
  auto add = [&](int cin, int cout) {
    Conv c;
    c.cin = cin;
    c.c8 = (cin + 7) / 8;
    c.cout = cout;
    c.woff = off;
    off += (size_t)cout * 9 * cin;
    c.boff = off;
    off += cout;
    return c;
  };
  enc_a_.resize(L_);
  enc_b_.resize(L_);
  dec_a_.resize(L_);
  dec_b_.resize(L_);
  int prev = 3;
  for (int l = 0; l < L_; ++l) {
    enc_a_[l] = add(prev, C_[l]);
    enc_b_[l] = add(C_[l], C_[l]);
    prev = C_[l];
  }
  for (int l = L_ - 2; l >= 0; --l) {
    dec_a_[l] = add(C_[l] + C_[l + 1], C_[l]);
    dec_b_[l] = add(C_[l], C_[l]);
  }
  head_off_ = off;
  np_ = off + 2 * (size_t)C_[0] + 2;
  w_ = alloc<float>(np_);
  g_ = alloc<float>(np_);
  m1_ = alloc<float>(np_);
  m2_ = alloc<float>(np_);
  eta_ = alloc<float>((size_t)m * m);
  if (eta_) cudaMemcpy(eta_, eta.data(), sizeof(float) * m * m, cudaMemcpyHostToDevice);
  auto packed = [&](Conv& c, bool back) {
    c.wf = alloc<unsigned char>(packed_weight_elems(c.cout, c.c8) * 2);
    if (back) c.wb = alloc<unsigned char>(packed_weight_elems(c.c8 * 8, c.cout / 8) * 2);
  };
  for (int l = 0; l < L_; ++l) {
    packed(enc_a_[l], l > 0);
    packed(enc_b_[l], true);
    if (l < L_ - 1) {
      packed(dec_a_[l], true);
      packed(dec_b_[l], true);
    }
  }
  // activations and gradients
  const size_t B = (size_t)bmax_;
  auto px = [&](int l) { return B * (size_t)(mp_ >> l) * (mp_ >> l); };
  x_ = alloc<__nv_bfloat16>(px(0) * 8);
  zea_.resize(L_);
  aea_.resize(L_);
  zeb_.resize(L_);
  cat_.assign(L_, nullptr);
  pool_.assign(L_, nullptr);
  zda_.assign(L_, nullptr);
  ada_.assign(L_, nullptr);
  zdb_.assign(L_, nullptr);
  out_.assign(L_, nullptr);
  gcat_.assign(L_, nullptr);
  gp_.assign(L_, nullptr);
  for (int l = 0; l < L_; ++l) {
    zea_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
    aea_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
    zeb_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
    if (l < L_ - 1) {
      cat_[l] = alloc<__nv_bfloat16>(px(l) * (C_[l] + C_[l + 1]));
      pool_[l] = alloc<__nv_bfloat16>(px(l + 1) * C_[l]);
      zda_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
      ada_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
      zdb_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
      out_[l] = alloc<__nv_bfloat16>(px(l) * C_[l]);
      gcat_[l] = alloc<float>(px(l) * (C_[l] + C_[l + 1]));
    }
    if (l > 0) gp_[l] = alloc<float>(px(l) * C_[l - 1]);
  }
  bottom_ = alloc<__nv_bfloat16>(px(L_ - 1) * C_[L_ - 1]);
  size_t gmax = 0;
  for (int l = 0; l < L_; ++l) gmax = std::max(gmax, px(l) * (size_t)C_[l]);
  gz_ = alloc<__nv_bfloat16>(gmax);
  ga_ = alloc<float>(gmax);
  gb_ = alloc<float>(gmax);
  glow_ = alloc<float>(gmax);
  head_out_ = alloc<float>(px(0) * 2);
  gout_ = alloc<float>(px(0) * 2);
  s_ = alloc<double>(B);
  num_ = alloc<double>(B);
  den_ = alloc<double>(B);
  // weight-gradient scratch: slices x cout x 9 x cin for the largest layer
  auto slices_for = [&](const Conv& c, int l) {
    const long long tiles = (long long)((c.cout + 15) / 16) * ((c.cin + 15) / 16);
    long long sl = std::max<long long>(1, 4 * 152 / tiles);
    sl = std::min<long long>(sl, std::max<long long>(1, (long long)px(l) / 256));
    return (int)std::min<long long>(sl, 128);
  };
  for (int l = 0; l < L_; ++l) {
    for (const Conv* c : {&enc_a_[l], &enc_b_[l], &dec_a_[l], &dec_b_[l]}) {
      if (l == L_ - 1 && (c == &dec_a_[l] || c == &dec_b_[l])) continue;
      wpart_n_ = std::max(wpart_n_, (size_t)slices_for(*c, l) * c->cout * 9 * c->cin);
    }
  }
  wpart_n_ = std::max(wpart_n_, (size_t)256 * 2 * (C_[0] + 1));
  wpart_ = alloc<float>(wpart_n_);
}

UNet::~UNet() {
  for (void* p : owned_) cudaFree(p);
}

int UNet::launches_per_forward() const {
  // per encoder level above the bottom: 2 convolutions + pooling; bottom: 2;
  // per decoder level: doubling + 2 convolutions; head; input (2) and output (1)
  return 6 * (L_ - 1) + 2 + 1 + 3;
}

cudaError_t UNet::pack(cudaStream_t s) {
  for (int l = 0; l < L_; ++l) {
    for (Conv* c : {&enc_a_[l], &enc_b_[l], &dec_a_[l], &dec_b_[l]}) {
      if (!c->wf) continue;
      UN_CU(launch_pack_weights(w_ + c->woff, reinterpret_cast<__nv_bfloat16*>(c->wf), c->cout, c->cin, c->c8, 0, s));
      if (c->wb)
        UN_CU(launch_pack_weights(w_ + c->woff, reinterpret_cast<__nv_bfloat16*>(c->wb), c->cout, c->cin, c->c8, 1,
                                  s));
    }
  }
  return cudaSuccess;
}

cudaError_t UNet::set_params(const float* host, cudaStream_t s) {
  UN_CU(cudaMemcpyAsync(w_, host, sizeof(float) * np_, cudaMemcpyHostToDevice, s));
  UN_CU(cudaMemsetAsync(m1_, 0, sizeof(float) * np_, s));
  UN_CU(cudaMemsetAsync(m2_, 0, sizeof(float) * np_, s));
  step_ = 0;
  UN_CU(pack(s));
  return cudaStreamSynchronize(s);
}

cudaError_t UNet::get_params(float* host, cudaStream_t s) {
  UN_CU(cudaMemcpyAsync(host, w_, sizeof(float) * np_, cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

cudaError_t UNet::conv(const Conv& c, int level, int B, const __nv_bfloat16* x, int xs, __nv_bfloat16* z,
                       __nv_bfloat16* act, int as, int ao, cudaStream_t s) {
  ConvArgs a{};
  a.x = x;
  a.xs = xs;
  a.xo = 0;
  a.w = c.wf;
  a.bias = w_ + c.boff;
  a.B = B;
  a.H = a.W = mp_ >> level;
  a.C8 = c.c8;
  a.nchunk = conv_chunks(c.c8);
  a.cout = c.cout;
  a.mode = 0;
  a.z = z;
  a.zs = c.cout;
  a.zo = 0;
  a.act = act;
  a.as = as;
  a.ao = ao;
  a.err = err_;
  return launch_conv_umma(a, s);
}

cudaError_t UNet::conv_back(const Conv& c, int level, int B, const __nv_bfloat16* gz, float* gx, cudaStream_t s) {
  ConvArgs a{};
  a.x = gz;
  a.xs = c.cout;
  a.xo = 0;
  a.w = c.wb;
  a.bias = nullptr;
  a.B = B;
  a.H = a.W = mp_ >> level;
  a.C8 = c.cout / 8;
  a.nchunk = conv_chunks(c.cout / 8);
  a.cout = c.c8 * 8;
  a.mode = 1;
  a.y = gx;
  a.ys = c.c8 * 8;
  a.yo = 0;
  a.err = err_;
  return launch_conv_umma(a, s);
}

cudaError_t UNet::wgrad(const Conv& c, int level, int B, const __nv_bfloat16* gz, const __nv_bfloat16* x, int xs,
                        cudaStream_t s) {
  WgradArgs a{};
  a.gz = gz;
  a.gs = c.cout;
  a.x = x;
  a.xs = xs;
  a.xo = 0;
  a.B = B;
  a.H = a.W = mp_ >> level;
  a.cout = c.cout;
  a.cin = c.cin;
  const long long npix = (long long)B * a.H * a.W;
  const long long tiles = (long long)((c.cout + 15) / 16) * ((c.cin + 15) / 16);
  long long sl = std::max<long long>(1, 4 * 152 / tiles);
  sl = std::min<long long>(sl, std::max<long long>(1, npix / 256));
  a.slices = (int)std::min<long long>(sl, 128);
  if ((size_t)a.slices * c.cout * 9 * c.cin > wpart_n_) return cudaErrorInvalidValue;
  a.part = wpart_;
  return launch_wgrad(a, g_ + c.woff, g_ + c.boff, gz, s);
}

cudaError_t UNet::forward(int B, cudaStream_t s) {
  for (int l = 0; l < L_; ++l) {
    const __nv_bfloat16* in = l == 0 ? x_ : pool_[l - 1];
    const int xs = l == 0 ? 8 : C_[l - 1];
    UN_CU(conv(enc_a_[l], l, B, in, xs, zea_[l], aea_[l], C_[l], 0, s));
    if (l < L_ - 1) {
      const int cs = C_[l] + C_[l + 1];
      UN_CU(conv(enc_b_[l], l, B, aea_[l], C_[l], zeb_[l], cat_[l], cs, 0, s));
      UN_CU(launch_avgpool2(cat_[l], cs, pool_[l], B, mp_ >> l, mp_ >> l, C_[l], s));
    } else {
      UN_CU(conv(enc_b_[l], l, B, aea_[l], C_[l], zeb_[l], bottom_, C_[l], 0, s));
    }
  }
  for (int l = L_ - 2; l >= 0; --l) {
    const int cs = C_[l] + C_[l + 1];
    const __nv_bfloat16* low = (l + 1 == L_ - 1) ? bottom_ : out_[l + 1];
    UN_CU(launch_up2(low, C_[l + 1], cat_[l], cs, C_[l], B, mp_ >> l, mp_ >> l, s));
    UN_CU(conv(dec_a_[l], l, B, cat_[l], cs, zda_[l], ada_[l], C_[l], 0, s));
    UN_CU(conv(dec_b_[l], l, B, ada_[l], C_[l], zdb_[l], out_[l], C_[l], 0, s));
  }
  return launch_head(out_[0], C_[0], w_ + head_off_, head_out_, (long long)B * mp_ * mp_, s);
}

cudaError_t UNet::backward(int B, cudaStream_t s) {
  const long long npix0 = (long long)B * mp_ * mp_;
  const int hs = (int)std::min<long long>(128, std::max<long long>(1, npix0 / 1024));
  UN_CU(launch_head_backward(gout_, out_[0], C_[0], w_ + head_off_, ga_, wpart_, g_ + head_off_, npix0, hs, s));
  const float* g = ga_;
  for (int l = 0; l < L_ - 1; ++l) {
    const int H = mp_ >> l, cs = C_[l] + C_[l + 1];
    GradActArgs ga{};
    ga.g = g;
    ga.gsd = C_[l];
    ga.z = zdb_[l];
    ga.zs = C_[l];
    ga.out = gz_;
    ga.B = B;
    ga.H = ga.W = H;
    ga.C = C_[l];
    UN_CU(launch_grad_act(ga, s));
    UN_CU(wgrad(dec_b_[l], l, B, gz_, ada_[l], C_[l], s));
    UN_CU(conv_back(dec_b_[l], l, B, gz_, gb_, s));
    ga.g = gb_;
    ga.z = zda_[l];
    UN_CU(launch_grad_act(ga, s));
    UN_CU(wgrad(dec_a_[l], l, B, gz_, cat_[l], cs, s));
    UN_CU(conv_back(dec_a_[l], l, B, gz_, gcat_[l], s));
    UN_CU(launch_up2_backward(gcat_[l], cs, C_[l], glow_, B, H, H, C_[l + 1], s));
    g = glow_;
  }
  for (int l = L_ - 1; l >= 0; --l) {
    const int H = mp_ >> l;
    GradActArgs ga{};
    if (l == L_ - 1) {
      ga.g = glow_;
      ga.gsd = C_[l];
    } else {
      ga.gp = gp_[l + 1];
      ga.gk = gcat_[l];
      ga.gks = C_[l] + C_[l + 1];
      ga.gko = 0;
    }
    ga.z = zeb_[l];
    ga.zs = C_[l];
    ga.out = gz_;
    ga.B = B;
    ga.H = ga.W = H;
    ga.C = C_[l];
    UN_CU(launch_grad_act(ga, s));
    UN_CU(wgrad(enc_b_[l], l, B, gz_, aea_[l], C_[l], s));
    UN_CU(conv_back(enc_b_[l], l, B, gz_, ga_, s));
    GradActArgs gb{};
    gb.g = ga_;
    gb.gsd = C_[l];
    gb.z = zea_[l];
    gb.zs = C_[l];
    gb.out = gz_;
    gb.B = B;
    gb.H = gb.W = H;
    gb.C = C_[l];
    UN_CU(launch_grad_act(gb, s));
    UN_CU(wgrad(enc_a_[l], l, B, gz_, l == 0 ? x_ : pool_[l - 1], l == 0 ? 8 : C_[l - 1], s));
    if (l > 0) UN_CU(conv_back(enc_a_[l], l, B, gz_, gp_[l], s));
  }
  return cudaSuccess;
}

cudaError_t UNet::forward_from(const float* x_dev, float* out_dev, int B, cudaStream_t s) {
  if (B < 1 || B > bmax_) return cudaErrorInvalidValue;
  UN_CU(launch_pack_input(x_dev, (long long)B * mp_ * mp_, x_, s));
  UN_CU(forward(B, s));
  return cudaMemcpyAsync(out_dev, head_out_, sizeof(float) * 2 * B * mp_ * mp_, cudaMemcpyDeviceToDevice, s);
}

cudaError_t UNet::backward_to(const float* gout_dev, float* grads_dev, int B, cudaStream_t s) {
  if (B < 1 || B > bmax_) return cudaErrorInvalidValue;
  UN_CU(cudaMemcpyAsync(gout_, gout_dev, sizeof(float) * 2 * B * mp_ * mp_, cudaMemcpyDeviceToDevice, s));
  UN_CU(backward(B, s));
  return cudaMemcpyAsync(grads_dev, g_, sizeof(float) * np_, cudaMemcpyDeviceToDevice, s);
}

cudaError_t UNet::train_step(const double2* rc, const double2* uc, int B, double lr, double* loss, cudaStream_t s) {
  if (B < 1 || B > bmax_) return cudaErrorInvalidValue;
  const long long ld = (long long)m_ * m_;
  UN_CU(launch_make_input<double2>(rc, ld, m_, mp_, B, eta_, s_, x_, s));
  UN_CU(forward(B, s));
  UN_CU(launch_loss(head_out_, uc, ld, s_, m_, mp_, B, num_, den_, gout_, s));
  UN_CU(backward(B, s));
  ++step_;
  const double b1 = 0.9, b2 = 0.999;
  UN_CU(launch_adam(w_, g_, m1_, m2_, (long long)np_, (float)lr, (float)b1, (float)b2,
                    (float)(1.0 - std::pow(b1, (double)step_)), (float)(1.0 - std::pow(b2, (double)step_)), 1e-8f, s));
  UN_CU(pack(s));
  if (loss) {
    std::vector<double> nu(B), de(B);
    UN_CU(cudaMemcpyAsync(nu.data(), num_, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    UN_CU(cudaMemcpyAsync(de.data(), den_, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    UN_CU(cudaStreamSynchronize(s));
    double acc = 0;
    for (int b = 0; b < B; ++b) acc += nu[b] / de[b];
    *loss = acc / B;
  }
  return cudaSuccess;
}

template <typename C>
cudaError_t UNet::correct(const C* rc, C* uc, long long ld, int B, cudaStream_t s) {
  for (int b0 = 0; b0 < B; b0 += bmax_) {
    const int nb = std::min(bmax_, B - b0);
    UN_CU(launch_make_input<C>(rc + (size_t)b0 * ld, ld, m_, mp_, nb, eta_, s_, x_, s));
    UN_CU(forward(nb, s));
    UN_CU(launch_write_correction<C>(head_out_, s_, m_, mp_, nb, uc + (size_t)b0 * ld, ld, s));
  }
  return cudaSuccess;
}
template cudaError_t UNet::correct<double2>(const double2*, double2*, long long, int, cudaStream_t);
template cudaError_t UNet::correct<float2>(const float2*, float2*, long long, int, cudaStream_t);

}  // namespace th
