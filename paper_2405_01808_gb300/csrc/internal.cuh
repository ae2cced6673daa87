// Internal definitions of the GB300 GRAND decoder library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "grand.h"

namespace grand {

constexpr int kSMax = GRAND_S_MAX;   // cut-off limit: 4^12 TEPs per frame
constexpr int kWMax = 16;            // syndrome words: N - K <= 512
constexpr int kNMax = GRAND_N_MAX;
constexpr int kLMax = 512;           // symbols per frame (N = 1024 with QPSK)
constexpr int kSideMax = 6;          // ranks per side of the search split (4^6 table entries)
constexpr int kTableMax = 4096;      // 4^kSideMax
constexpr uint16_t kNoPos = 0xFFFF;  // alternative bit beyond N (padding): no syndrome change

// Device view of one code: column-packed parity-check matrix.
//   hcol[j * W + w] bit b = H[32 w + b][j]   (column j of H, W words)
//   hf[j] = XOR of p_r over the rows r with H[r][j] = 1, for fixed
//           pseudo-random 32-bit words p_r: a random linear projection of
//           column j. The projection of a syndrome is the XOR of hf over the
//           flipped positions; a zero syndrome has a zero projection, so it
//           is a filter in front of the full test (false matches ~ 2^-32).
//   polar: every row r of H is column frozen[r] of G_N = F^{(x)n} (Def. II.1),
//          so H y is the frozen part of the polar transform y G_N and the
//          preparation computes it with log2 N butterfly stages instead of
//          column loads; prow[r] = p_r (the projection word of row r).
//   hrow[r * (N/32) + w] bit b = H[r][32 w + b]   (row r of H, as given to
//          grand_code_create): the row-parity membership test.
//   status[0]: set (atomicOr 1) by a kernel that cut a frame at the call's
//          deadline; status[1]: where grand_stream_status takes it to.
struct CodeDev {
  const uint32_t* hcol;
  const uint32_t* hf;
  const uint16_t* frozen;
  const uint32_t* prow;
  const uint32_t* hrow;
  uint32_t* status;
  int32_t N, K, R, W;
  int32_t polar;
};

// Per-frame state handed from the preparation kernel to the search kernel
// for frames the preparation could not finish.
struct FrameRec {
  uint32_t frame;            // frame index in the batch
  uint16_t code;             // index into the code table
  uint8_t sp;                // S' = min(S, L)
  uint8_t w_done;            // every TEP with at most w_done altered symbols was tested
  int64_t cw_off;            // first output word of the frame
  uint32_t s0[kWMax];        // base syndrome H y
  uint16_t pos[kSMax][2];    // bit position flipped by the I / Q alternative of rank r
  uint8_t ex[kSMax];         // bit0 h exists, bit1 v exists, bit2 diag exists
  uint32_t f0;               // projection of s0 (see CodeDev::hf)
};
static_assert(sizeof(FrameRec) % 8 == 0, "FrameRec alignment");

// Scratch shared by the kernels of one decode call (device memory).
struct Scratch {
  unsigned int n_hard;              // frames appended by the preparation kernel
  unsigned int next;                // search work-queue head
  unsigned long long evaluated;     // TEP checks executed
  unsigned long long search_useful; // valid queries answered by the search stage
  unsigned long long t0;            // %globaltimer at the call's first look at the clock (deadline)
};

// Per-TEP decode (five-point NNE order, or a membership test other than the
// split search): defined in per_tep.cu, called by grand_decode_symbols after
// its argument checks.
int run_per_tep(const grand_code* c, const grand_params* p, const void* symbols, int64_t n_frames, uint32_t* cw,
                uint32_t* queries, uint8_t* abandon, grand_stats* stats, cudaStream_t st);

// Load every kernel of the symbol-level decode now (the serving loop calls it
// at creation so that no batch pays a lazy module load).
int preload_qam_kernels();

// grand_decode_mixed on a code table already resident on the device (the
// serving loop keeps one for its lifetime). The caller has validated params
// (QAM order, membership AUTO or HASH); Lmax / Wmax bound L and W over the
// table. w_step > 0 with cursors: the resumable search (frames with no hit in
// the first w_step weights beyond the preparation's get abandon 6 and their
// cursor at cursors[frame]).
int decode_mixed_resident(const CodeDev* d_table, int n_codes, int Lmax, int Wmax, const grand_params* p,
                          const grand_frame_desc* desc, int64_t n_frames, const void* symbols, int64_t n_symbols,
                          uint32_t* cw, int64_t n_cw_words, uint32_t* queries, uint8_t* abandon, cudaStream_t st,
                          int w_step = 0, FrameRec* cursors = nullptr);

// The next weight window of every suspended cursor (abandon 6) of
// cursors[0..n): cursor i writes its outputs at queries[i], abandon[i] and
// cw + i * cw_stride, and stays suspended (with its w_done advanced) when the
// window holds no codeword and weights below the cap remain.
int resume_resident(const CodeDev* d_table, int n_codes, int Wmax, const grand_params* p, FrameRec* cursors,
                    int64_t n, int w_step, uint32_t* cw, int64_t cw_stride, uint32_t* queries, uint8_t* abandon,
                    cudaStream_t st);

}  // namespace grand

// Opaque code object of the ABI.
struct grand_code {
  int N, K, R, W;
  uint32_t* d_hcol;                 // device, N * W words, then the N projections hf
  grand::CodeDev* d_dev;            // device copy of the CodeDev (for code tables)
  uint32_t* d_status;               // device, 2 words (CodeDev::status)
  grand::CodeDev dev;               // host copy of the device view
  int device;                       // CUDA device the object lives on
};
