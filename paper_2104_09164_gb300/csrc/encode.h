// encode.h -- host-side CKKS encoding / decoding and CRT lift.
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>
#include "hostmath.h"

namespace hear {

struct EncoderTables;
std::shared_ptr<EncoderTables> make_encoder_tables(uint32_t log_n);
// round(scale * tau^-1(z)) for N/2 real slots; returns the number of near-ties (|frac-1/2| < 2^-30)
int encode_dd(const EncoderTables &T, const double *z, double scale, int64_t *m_out);
// count vectors of N/2 slots each, in parallel on the host cores
void encode_many(const EncoderTables &T, const double *z, size_t count, const double *scales, int64_t *m_out);
// slot values from N real coefficients (already divided by the scale)
void decode_double(uint32_t log_n, const double *v, double *z);
// centred CRT lift of residues [L1][N] times inv_scale
void crt_to_double(const uint64_t *res, const uint64_t *primes, uint32_t L1, uint32_t n, double inv_scale,
                   double *out);

}  // namespace hear
