// Host-side check of the tensor-core Gram's shared-memory arithmetic: the
// bank pattern of the operand stores, the furthest byte any MMA operand read
// reaches for both tile parities, and the descriptor bit fields.  Runs on the
// CPU; no kernel is launched.
#include <cstdio>

#include "gram_tc.cuh"

using namespace ntc;

template <int VT, int NT>
static int check() {
    using G = GramTC<4, VT, 1, NT>;
    int bad_banks = 0;
    // product(): slot j of thread tid is visit v = (tid + j NT) / SPV, ranks
    // 8q .. 8q + 7 with q = tid % SPV; rank 8q + c of part (0 big, 1 small) at
    // S + q SBO + (v / 4) KGB + (v % 4) 4 + c 16 + part 4 SBO
    for (int warp = 0; warp < NT / 32; ++warp)
        for (int j = 0; j < G::RS; ++j)
            for (int c = 0; c < 8; ++c)
                for (int part = 0; part < 2; ++part)
                    for (int buf = 0; buf < 2; ++buf) {
                        int hits[32] = {0};
                        for (int lane = 0; lane < 32; ++lane) {
                            const int tid = 32 * warp + lane, q = tid % G::SPV, v = (tid + j * NT) / G::SPV;
                            const int byte = G::S_OFF + buf * G::SB + q * G::SBO + (v >> 2) * G::KGB + (v & 3) * 4 +
                                             c * 16 + part * 4 * G::SBO;
                            if (byte < G::S_OFF + buf * G::SB || byte + 4 > G::S_OFF + (buf + 1) * G::SB) {
                                std::printf("store outside its buffer\n");
                                return 1;
                            }
                            ++hits[(byte / 4) % 32];
                        }
                        for (int b = 0; b < 32; ++b) bad_banks += hits[b] > 1;
                    }
    // MMA operand reads: tile parity p uses buffer p; A (M = 128 rows) starts
    // 8 SBO early for odd tiles, B (N rows) at the buffer; each K step reads two
    // 16-byte core-matrix columns KGB apart, 8-row groups SBO apart
    long lo = 1L << 40, hi = -1;
    for (int p = 0; p < 2; ++p)
        for (int ks = 0; ks < VT / 8; ++ks) {
            const long base = G::S_OFF + p * G::SB + ks * 2 * G::KGB;
            const long astart = base - (p ? 8 * G::SBO : 0);
            for (int row = 0; row < G::M; ++row)
                for (int kc = 0; kc < 2; ++kc) {
                    const long a = astart + (row / 8) * G::SBO + (row % 8) * 16 + kc * G::KGB;
                    lo = a < lo ? a : lo;
                    hi = a + 16 > hi ? a + 16 : hi;
                }
            for (int row = 0; row < G::N; ++row)
                for (int kc = 0; kc < 2; ++kc) {
                    const long b = base + (row / 8) * G::SBO + (row % 8) * 16 + kc * G::KGB;
                    lo = b < lo ? b : lo;
                    hi = b + 16 > hi ? b + 16 : hi;
                }
        }
    // the useful rows of A: S rows 0..63 of the tile's own buffer
    int rows_ok = 1;
    for (int p = 0; p < 2; ++p)
        for (int row = 0; row < 2 * G::RP; ++row) {
            const int arow = row + (p ? 64 : 0);
            const long a = (G::S_OFF + p * G::SB - (p ? 8 * G::SBO : 0)) + (arow / 8) * G::SBO + (arow % 8) * 16;
            const long want = G::S_OFF + p * G::SB + (row / 8) * G::SBO + (row % 8) * 16;
            rows_ok &= a == want;
        }
    // descriptor fields
    const uint64_t d = tc::smem_desc(0x1230u, (uint32_t)G::KGB, (uint32_t)G::SBO);
    const int desc_ok = ((d & 0x3FFF) << 4) == 0x1230u && (((d >> 16) & 0x3FFF) << 4) == (uint64_t)G::KGB &&
                        (((d >> 32) & 0x3FFF) << 4) == (uint64_t)G::SBO && ((d >> 46) & 3) == 1 && (d >> 61) == 0;
    const uint32_t id = G::IDESC;
    const int idesc_ok = ((id >> 4) & 3) == 1 && ((id >> 7) & 7) == 2 && ((id >> 10) & 7) == 2 &&
                         ((id >> 15) & 3) == 0 && ((id >> 17) & 63) == (uint32_t)(G::N >> 3) &&
                         ((id >> 24) & 31) == (uint32_t)(G::M >> 4);
    // the M = 64 form of the split-row kernel: same fields, M / 16 = 4
    const uint32_t id64 = G::IDESC64;
    const int idesc64_ok = (id64 & ~(31u << 24)) == (id & ~(31u << 24)) && ((id64 >> 24) & 31) == 4u;
    const int epi = 4 * G::RP * G::TSTR * 4 + NT * 32;
    std::printf("VT %d NT %d bytes %d sb %d kgb %d sbo %d bank_conflicts %d read_lo %ld read_hi %ld rows_ok %d "
                "desc_ok %d idesc_ok %d idesc64_ok %d epilogue %d tcols %d blocks %d\n",
                VT, NT, G::BYTES, G::SB, G::KGB, G::SBO, bad_banks, lo, hi, rows_ok, desc_ok, idesc_ok, idesc64_ok, epi,
                G::TCOLS, G::BLOCKS);
    return 0;
}

int main() {
    int rc = check<64, 128>();
    rc |= check<64, 256>();
    return rc;
}
