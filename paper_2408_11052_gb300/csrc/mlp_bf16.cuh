// BF16 tensor-core MLP (encoders phi, psi and the policy pi): buffers and entry points.
//
// Every product is a GEMM on tcgen05 (BF16 in, FP32 accumulate in TMEM),
// each operand read as it is stored:
//   forward      z_l  = h_{l-1} W_l^T          A = h_{l-1} [M][K],      B = W_l  [N][K]   (K-major)
//   input grad   dh   = dz_l W_l               A = dz_l    [M][N],      B = Wt_l [K][N]   (K-major)
//   weight grad  dW_l = dz_l^T [h_{l-1} | 1]   A = dz_l    [batch][out], B = [h | 1] [batch][in + 1]
//                                              (both MN-major: the batch is K)
// The column of ones after h's hi part (after x0's split input) makes the
// weight-gradient GEMM return the bias gradient (sum over the batch) as its
// last column; no activation or gradient is stored twice.
//
// The network input (observations, actions, goals: O(1..10) values with a
// large common component across the batch) is split into a BF16 high part and
// a BF16 residual, interleaved along K (x0 = [hi_0, lo_0, hi_1, lo_1, ...]),
// with the first-layer weight shadow duplicated to match ([w_0, w_0, w_1, ...]):
// the first product then sees the input with ~16 mantissa bits.  Rounding the
// raw input to plain BF16 was the dominant error of the BF16 path (gradient
// cosine 0.992 instead of 0.9998 on small batches).
//
// Forward products use the weights as a BF16 pair W = W_hi + W_lo (W_lo =
// bf16(W - W_hi)).  Rounding the weights to a single BF16 was the next largest
// error (first-layer weight-gradient cosine 0.998 on 96-wide networks; 0.9993+
// with the pair).  Hidden activations are kept as a BF16 pair too, h = h_hi +
// h_lo, and the later layers take three products, h_hi W_hi + h_lo W_hi +
// h_hi W_lo (A = [h_hi | h_lo] against B = [W_hi | W_hi | W_lo], the A slices
// wrapping around): a single BF16 h moves about 0.05 % of the ReLU decisions
// of a 4 x 1024 LayerNorm encoder to the other side of zero compared with FP64
// (CPU emulation: 2247 of 4.2 M units, first-layer weight-gradient cosine
// 0.9978), the pair about 1e-6 (5 units, cosine 0.999998).  The backward uses
// single BF16 shadows Wt [in][out] and the hi part of h (its rounding hardly
// moves the gradient).
// The backward epilogue likewise writes dz and dz^T.  The shadows are refreshed
// from the FP32 master weights before each step.
//
// The same layer of several networks (phi and psi; pi and psi) runs as one
// grouped launch, and the weight gradients of all layers run as one launch
// after the input-gradient chain (they are off its critical path).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "tables.h"
#include "tc_gemm.cuh"

namespace crl {

constexpr int kMaxGroupNets = 4;

struct BfLayer {
  int in, out, in_pad, out_pad;   // in_pad: row length of W, (nhi + 1) kp; out_pad: multiple of 8
  int kin;                        // K of one product: in, or 2 in for the split first layer
  int kp;                         // kin rounded up to 64
  int nhi;                        // copies of W_hi before W_lo: 1 (first layer), 2 (later layers)
  int64_t oW, ob, og, obeta;      // offsets into the FP32 master array (og/obeta < 0: no LayerNorm)
  __nv_bfloat16* W;               // [out][in_pad]: first layer [W_hi | W_lo] (columns duplicated for the
                                  // split input); later layers [W_hi | W_hi | W_lo] for A = [h_hi | h_lo]
  __nv_bfloat16* Wt;              // [in][out_pad]
  CUtensorMap tmW, tmWt;
  // split-K of the weight-gradient product (K = the batch): partial tiles and
  // per-tile tickets, for batches large enough to split (wsplit_cap > 1)
  int wsplit_cap;
  float* wpart;
  unsigned* wtick;
};

// One network's BF16 state for batches of up to Mmax rows.
struct BfNet {
  MlpShape s;
  int Mmax = 0;
  int layers = 0;
  BfLayer L[CRL_MAX_LAYERS + 1];
  // activations
  // The weight-gradient products read x0 and h as MN-major operands (the
  // batch is their K), so no transposed copy exists; the bias gradient comes
  // from a column of ones after the hi part (x0: column 2 in, h: column H).
  __nv_bfloat16* x0 = nullptr;    // [Mmax][pad8(2 in + 1)] split input (hi, lo interleaved), then ones
  int ldh = 0;                    // row length of h: 2 kp(H) + 128
  int hlo = 0;                    // column of h_lo: kp(H) + 128 (columns H .. hlo - 1: the ones column
                                  // H, zeros elsewhere; the forward skips the 128 columns at kp(H))
  __nv_bfloat16* h[CRL_MAX_LAYERS] = {};   // [Mmax][ldh] BF16 hi part [0, H) and lo part [hlo, hlo + H)
  float* z[CRL_MAX_LAYERS] = {};           // LayerNorm: pre-norm [Mmax][H], then zhat in place
  float* rstd[CRL_MAX_LAYERS] = {};        // LayerNorm: [Mmax]
  float* y = nullptr;                      // [Mmax][out] output (FP32)
  // backward: dz[l] = gradient at the output of layer l (pre-activation of a
  // hidden layer, y for l = layers), BF16 [Mmax][ld] with ld = H (hidden) or
  // out_pad (output)
  __nv_bfloat16* dz[CRL_MAX_LAYERS + 1] = {};
  float* du = nullptr;                     // LayerNorm backward input [Mmax][H]
  float* ln_partial = nullptr;             // LayerNorm gain / shift gradient block sums [layers][Mmax/8][2][H]
  // tensor maps, built for the batch size M of the last call
  int tm_M = -1;
  CUtensorMap tm_x0A, tm_x0B;    // A of the first layer; MN-major B of its weight gradient (2 in + 1 columns)
  CUtensorMap tm_hA[CRL_MAX_LAYERS], tm_hB[CRL_MAX_LAYERS];   // the same for h (H + 1 columns)
  CUtensorMap tm_dzA[CRL_MAX_LAYERS + 1];   // K-major A of the input gradient, MN-major A of the weight gradient
};

// Device problem tables of the grouped GEMM, one per distinct list of problems
// (keyed by content: tensor maps, sizes and epilogue pointers).  A table is
// written once, before its first launch, and never changed, so a captured
// CUDA graph may keep replaying it.  Building a table is a synchronous copy:
// it must not happen while the stream is being captured.
class GemmGroups {
 public:
  GemmGroups() = default;
  GemmGroups(const GemmGroups&) = delete;
  GemmGroups& operator=(const GemmGroups&) = delete;
  ~GemmGroups() { reset(); }
  // Fills tiles_n / tile_begin of `probs` for tile width BN and returns the
  // device table; nullptr (and *err) on failure.
  // BN = 0: the problems are uploaded as given (tiles_n / tile_begin untouched).
  // allow_split: problems with ksplit_cap > 1 split K (the one-tile kernel
  // only) so that the launch has about two CTAs per SM.  BM: tile rows (128,
  // or 256 for the CTA-pair kernel).
  const tc::GemmProblem* table(std::vector<tc::GemmProblem>& probs, int BN, int* total_tiles, cudaStream_t st,
                               const char** err, bool allow_split = false, int BM = tc::kBM);
  // Frees every table (synchronises the device) and forgets the tuned tile widths.
  void reset();
  // Autotuned configuration (8192 x kernel + 16 x tile width + ring depth) of a problem list,
  // keyed by its untiled content; 0 if none.
  int tuned_bn(uint64_t key) const {
    auto it = tuned_.find(key);
    return it == tuned_.end() ? 0 : it->second;
  }
  void set_tuned_bn(uint64_t key, int cfg) { tuned_[key] = cfg; }
  // What the autotuner measured for one problem list (crl_gemm_tuning_report).
  struct TuneRecord {
    int nprob;
    int M0, N0, K0;          // the list's first problem
    double flops;            // algorithmic work of one launch
    double issued;           // tensor work as launched: sum of 2 M N K over the problems, K counting
                             // every BF16 product (hi / lo input and weight pairs)
    int cfg;                 // the configuration kept
    int ncand;
    int cand[16];            // candidate configurations, in the order timed
    float us[16];            // their best time per launch over the timing rounds
  };
  void add_record(const TuneRecord& r) { records_.push_back(r); }
  const std::vector<TuneRecord>& records() const { return records_; }
  // Number of distinct problem lists with a device table.
  size_t entries() const { return map_.size(); }
  // false: never time candidates (fixed rule), for problem lists that change
  // with every call (the op-level entry points on caller workspaces).
  bool allow_tune = true;

 private:
  std::unordered_map<uint64_t, int> tuned_;
  std::vector<TuneRecord> records_;
  struct Entry {
    const tc::GemmProblem* dev;
    int tiles;
    std::vector<tc::GemmProblem> host;
  };
  std::unordered_map<uint64_t, std::vector<Entry>> map_;
  std::vector<void*> chunks_;
  tc::GemmProblem* cur_ = nullptr;
  int used_ = 0, cap_ = 0;
};

// Allocates the network's BF16 buffers (cudaMalloc through `alloc`) and writes the ones rows.
// Returns an error message or nullptr.
using DevAlloc = void* (*)(void* owner, size_t bytes);
const char* bf_net_init(BfNet& n, const MlpShape& s, int Mmax, DevAlloc alloc, void* owner);
// Only the pointer assignment of bf_net_init (and, with weight_maps, the
// weight shadows' tensor maps): no memory is touched.
const char* bf_net_carve(BfNet& n, const MlpShape& s, int Mmax, DevAlloc alloc, void* owner, bool weight_maps);
// Bytes bf_net_carve takes for Mmax rows (256-byte aligned pieces).
size_t bf_net_bytes(const MlpShape& s, int Mmax);
// Writes the ones columns of x0 and every h on stream st.
void bf_net_fill_ones(BfNet& n, cudaStream_t st);
// (Re)build the activation tensor maps for batch M (no-op when M is unchanged).
const char* bf_net_maps(BfNet& n, int M);
// Refresh W / Wt shadows from the FP32 master parameters.
void bf_net_shadow(BfNet& n, const float* params, cudaStream_t st);
// Row length of x0 (the split input and the ones column): pad8(2 in + 1).
int bf_net_x0_ld(const BfNet& n);
// Pack the FP32 input concat(x0 [M][in0], x1 [M][in1]) into x0.
void bf_net_pack_input(BfNet& n, const float* x0, const float* x1, int M, cudaStream_t st);
// Store an FP32 gradient dy [M][out] into dz[layers] (BF16).
void bf_net_load_dy(BfNet& n, const float* dy, int M, cudaStream_t st);

// The fused energy's BF16 operand written by an encoder's output layer (see
// kEpiFwdOutEnergy): x [M][out], aux [M].
struct EnergyOut {
  __nv_bfloat16* X;
  float* aux;
  int energy;
};

// One network of a grouped pass.  All networks of a group have the same
// number of layers and the same hidden width and LayerNorm setting.
struct BfPass {
  BfNet* net;
  const float* params;
  float* grads;   // backward: FP32 gradients in the flat layout, or null (no weight gradients)
  float* dx1;     // backward: FP32 gradient of input columns [in0, in0 + in1) as [M][in1], or null
  int M;          // batch rows of this network (its tensor maps built for M)
  const EnergyOut* energy_out = nullptr;   // forward: also write the fused energy's operand
  float* dx0 = nullptr;   // backward: FP32 gradient of input columns [0, in0) as [M][in0], or null
};
// Forward of `count` networks (one grouped launch per layer): y [M][out] FP32 in net->y.
const char* bf_forward(GemmGroups& gg, const BfPass* nets, int count, unsigned* status, cudaStream_t st);
// Backward of `count` networks from their dz[layers]: one grouped
// input-gradient launch per hidden layer, then one launch with every weight
// gradient and first-layer input gradient.
const char* bf_backward(GemmGroups& gg, const BfPass* nets, int count, unsigned* status, cudaStream_t st);
// The autotuner's measurements of every problem list tuned in `gg`, as a JSON
// array (crl_gemm_tuning_report).
std::string gemm_tuning_json(const GemmGroups& gg);

// Adam on the FP32 master parameters of several networks in one launch, also
// refreshing each network's BF16 shadows (W_hi / W_lo and Wt) from the updated
// weights.  grads / m / v share the flat layout of params.
struct AdamShadowNet {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t n;
  const int* t_dev;   // Adam step counter (already incremented for this step)
  float lr, b1, b2, eps;
  BfNet* net;
};
// One launch for `count` networks (any number); its launch tables live in `cache`.
// heads: actor-head forwards run by extra blocks of the same launch (optional).
const char* adam_shadow_update(BlobCache& cache, const AdamShadowNet* nets, int count, cudaStream_t st,
                               const std::vector<HeadFwdArgs<float>>* heads = nullptr);

}  // namespace crl
