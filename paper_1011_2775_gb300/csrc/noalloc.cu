// mg_apply_noalloc: the fine-level operators of mg_apply without any device
// allocation, for callers that cannot call cudaMalloc themselves or through
// the library (see include/mgclover.h).  Its scratch -- the packed input and
// output halves and the two half-vector temporaries of D_r -- lives in one
// file-scope device array of fixed size, shared by every call.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoallocMaxSites = 16384;
// FP64 worst case: 6 half vectors (input even/odd, output even/odd, two
// temporaries) x 24 doubles x Vh = 576 bytes per site
constexpr size_t kNoallocScratchBytes = (size_t)kNoallocMaxSites * 576;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), resolved once
// per device.  In host code the array's name is only a host-side stand-in.
void* scratch_on(int device) {
  if (device < 0 || device >= kMaxDevices) mg::raise(MG_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      mg::raise(MG_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  return g_noalloc_ptr[device];
}

template <typename T>
void run_op(mg::Ctx* c, int op, T* base) {
  const mg::Geom& g = c->g;
  const size_t h = 24 * c->Vh;  // reals per half vector
  T* ie = base;
  T* io = base + h;
  T* oe = base + 2 * h;
  T* oo = base + 3 * h;
  T* t1 = base + 4 * h;
  T* t2 = base + 5 * h;
  cudaStream_t s = c->stream;
  switch (op) {
    case MG_OP_D:
      mg::dslash<T>(g, mg::EPI_CX_PAY, 0, oe, io, c->gauge<T>(), c->A<T>(0), ie, 1.0, 0xff, s);
      mg::dslash<T>(g, mg::EPI_CX_PAY, 1, oo, ie, c->gauge<T>(), c->A<T>(1), io, 1.0, 0xff, s);
      c->dslash_launches += 2;
      break;
    case MG_OP_DP:
      mg::clover_apply<T>(g, t1, ie, c->Ainv<T>(0), s);
      mg::clover_apply<T>(g, t2, io, c->Ainv<T>(1), s);
      mg::dslash<T>(g, mg::EPI_XPAY, 0, oe, t2, c->gauge<T>(), nullptr, ie, 1.0, 0xff, s);
      mg::dslash<T>(g, mg::EPI_XPAY, 1, oo, t1, c->gauge<T>(), nullptr, io, 1.0, 0xff, s);
      c->dslash_launches += 2;
      break;
    case MG_OP_DR:
      mg::clover_apply<T>(g, t1, ie, c->Ainv<T>(0), s);
      mg::dslash<T>(g, mg::EPI_CH, 1, t2, t1, c->gauge<T>(), c->Ainv<T>(1), nullptr, 0.0, 0xff, s);
      mg::dslash<T>(g, mg::EPI_XPAY, 0, oe, t2, c->gauge<T>(), nullptr, ie, -1.0, 0xff, s);
      c->dslash_launches += 2;
      MG_CUDA(cudaMemsetAsync(oo, 0, sizeof(T) * h, s));  // the array keeps the last call's contents
      break;
    case MG_OP_BR:
      mg::clover_apply<T>(g, t1, io, c->Ainv<T>(1), s);
      mg::dslash<T>(g, mg::EPI_XPAY, 0, oe, t1, c->gauge<T>(), nullptr, ie, -1.0, 0xff, s);
      c->dslash_launches += 1;
      MG_CUDA(cudaMemsetAsync(oo, 0, sizeof(T) * h, s));
      break;
    case MG_OP_M:
    case MG_OP_MINV: {
      const bool inv = op == MG_OP_MINV;
      mg::clover_apply<T>(g, oe, ie, inv ? c->Ainv<T>(0) : c->A<T>(0), s);
      mg::clover_apply<T>(g, oo, io, inv ? c->Ainv<T>(1) : c->A<T>(1), s);
      break;
    }
    case MG_OP_HOP:
      mg::dslash<T>(g, mg::EPI_H, 0, oe, io, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, s);
      mg::dslash<T>(g, mg::EPI_H, 1, oo, ie, c->gauge<T>(), nullptr, nullptr, 0.0, 0xff, s);
      c->dslash_launches += 2;
      break;
    default:
      mg::raise(MG_ERR_ARG, "mg_apply_noalloc supports D, D_p, D_r, b_r, M, M^{-1} and H on the fine level");
  }
}

}  // namespace

namespace mg {
void set_last_error(const std::string& what);
}

extern "C" int mg_apply_noalloc(void* ctx, int op, void* out, const void* in, int prec) {
  mg::set_last_error("");
  try {
    if (!ctx || !out || !in) mg::raise(MG_ERR_ARG, "null argument");
    mg::Ctx* c = static_cast<mg::Ctx*>(ctx);
    MG_CUDA(cudaSetDevice(c->device));
    if (prec != MG_FP64 && prec != MG_FP32) mg::raise(MG_ERR_ARG, "bad precision");
    if (!c->have_clover) mg::raise(MG_ERR_STATE, "set the gauge field and clover first");
    if (c->V > (size_t)kNoallocMaxSites)
      mg::raise(MG_ERR_DIMS, "mg_apply_noalloc is limited to lattices of at most 16384 sites");
    void* scratch = scratch_on(c->device);
    const bool f32 = prec == MG_FP32;
    const size_t h = 24 * c->Vh;
    if (f32) {
      float* base = static_cast<float*>(scratch);
      mg::pack_spinor(c->g, static_cast<const double*>(in), base, base + h, true, c->stream);
      run_op<float>(c, op, base);
      mg::unpack_spinor(c->g, base + 2 * h, base + 3 * h, true, static_cast<double*>(out), c->stream);
    } else {
      double* base = static_cast<double*>(scratch);
      mg::pack_spinor(c->g, static_cast<const double*>(in), base, base + h, false, c->stream);
      run_op<double>(c, op, base);
      mg::unpack_spinor(c->g, base + 2 * h, base + 3 * h, false, static_cast<double*>(out), c->stream);
    }
    c->sync();
    return MG_OK;
  } catch (const mg::Error& e) {
    mg::set_last_error(e.what);
    return e.code;
  } catch (...) {
    mg::set_last_error("unexpected error");
    return MG_ERR_CUDA;
  }
}
