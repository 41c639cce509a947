/*
 * opcount.cpp -- the oracle (mhd_oracle.c) compiled with an
 * operation-counting scalar in place of double.
 *
 * TEST / MEASUREMENT INFRASTRUCTURE ONLY: it gives the algorithmic
 * floating-point operation counts of each stage of the advance (and of the
 * CFL reduction) on a given input, for the ALU roofline of the GPU kernels.
 * Every +, -, *, / and sqrt of the oracle's arithmetic is counted once, in
 * the stage that the oracle's ORC_STAGE markers say is running; comparisons
 * (and so min / max and the limiter's sign tests) are counted apart; sign
 * flips and fabs are free.  The values computed are the oracle's own.
 * Single-threaded (OpenMP pragmas are ignored), so the counts are exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace opc {
enum { ADD, MUL, DIV, SQRT, CMP, NOPS };
constexpr int kStages = 16;
static int64_t count[kStages][NOPS];
static int stage = 0;
inline void tick(int op) { ++count[stage][op]; }
}  // namespace opc

struct ocnt {
  double v;
  ocnt() = default;
  ocnt(double x) : v(x) {}
  explicit operator double() const { return v; }
  ocnt& operator+=(ocnt b) { opc::tick(opc::ADD); v += b.v; return *this; }
  ocnt& operator-=(ocnt b) { opc::tick(opc::ADD); v -= b.v; return *this; }
  ocnt& operator*=(ocnt b) { opc::tick(opc::MUL); v *= b.v; return *this; }
  ocnt& operator/=(ocnt b) { opc::tick(opc::DIV); v /= b.v; return *this; }
};

inline ocnt operator+(ocnt a, ocnt b) { opc::tick(opc::ADD); return ocnt(a.v + b.v); }
inline ocnt operator-(ocnt a, ocnt b) { opc::tick(opc::ADD); return ocnt(a.v - b.v); }
inline ocnt operator*(ocnt a, ocnt b) { opc::tick(opc::MUL); return ocnt(a.v * b.v); }
inline ocnt operator/(ocnt a, ocnt b) { opc::tick(opc::DIV); return ocnt(a.v / b.v); }
inline ocnt operator-(ocnt a) { return ocnt(-a.v); }
inline ocnt operator+(ocnt a) { return a; }
inline bool operator<(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v < b.v; }
inline bool operator>(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v > b.v; }
inline bool operator<=(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v <= b.v; }
inline bool operator>=(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v >= b.v; }
inline bool operator==(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v == b.v; }
inline bool operator!=(ocnt a, ocnt b) { opc::tick(opc::CMP); return a.v != b.v; }
inline ocnt sqrt(ocnt a) { opc::tick(opc::SQRT); return ocnt(::sqrt(a.v)); }
inline ocnt fabs(ocnt a) { return ocnt(::fabs(a.v)); }

static_assert(sizeof(ocnt) == sizeof(double), "ocnt must have the layout of double");

#define double ocnt
#define ORC_STAGE(k) (opc::stage = (k))
extern "C" {
#include "mhd_oracle.c"
}
#undef double

extern "C" __attribute__((visibility("default"))) void opc_reset(void) {
  memset(opc::count, 0, sizeof opc::count);
  opc::stage = 0;
}

/* out: kStages x NOPS counts (add/sub, mul, div, sqrt, compare) per stage. */
extern "C" __attribute__((visibility("default"))) void opc_read(int64_t *out) {
  memcpy(out, opc::count, sizeof opc::count);
}

extern "C" __attribute__((visibility("default"))) int32_t opc_shape(int32_t *nops) {
  *nops = opc::NOPS;
  return opc::kStages;
}
