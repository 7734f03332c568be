// Host check of dpg::pk_word_ok (the join kernels' key check of one row
// word) against the definition it implements: every byte of word w that lies
// inside the 8-byte little-endian key at row byte pk_off equals that key
// byte.  All word sizes, every word that overlaps the key, key offsets
// 0..79, matching words and words with one flipped bit.  Exit status 0 when
// all cases agree.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "dpg_device.cuh"

template <int WB>
static bool by_bytes(const typename dpg::WordT<WB>::T& v, uint32_t w, uint32_t pk_off, uint64_t key) {
  uint8_t b[WB];
  std::memcpy(b, &v, WB);
  for (int j = 0; j < WB; ++j) {
    const uint32_t pos = w * WB + j;
    if (pos >= pk_off && pos < pk_off + 8 && b[j] != (uint8_t)(key >> (8 * (pos - pk_off)))) return false;
  }
  return true;
}

template <int WB>
static long check(std::mt19937_64& g) {
  long mismatches = 0, cases = 0;
  for (uint32_t pk = 0; pk < 80; ++pk)
    for (uint32_t w = 0; w * WB < pk + 8; ++w) {
      if (w * WB + WB <= pk) continue;  // the word ends before the key
      for (int t = 0; t < 400; ++t) {
        const uint64_t key = g();
        uint8_t b[16];
        for (int j = 0; j < 16; ++j) b[j] = (uint8_t)g();
        for (int j = 0; j < WB; ++j) {
          const uint32_t pos = w * WB + j;
          if (pos >= pk && pos < pk + 8) b[j] = (uint8_t)(key >> (8 * (pos - pk)));
        }
        if (t % 2) b[g() % WB] ^= (uint8_t)(1u << (g() % 8));
        typename dpg::WordT<WB>::T v;
        std::memcpy(&v, b, WB);
        mismatches += dpg::pk_word_ok<WB>(v, w, pk, key) != by_bytes<WB>(v, w, pk, key);
        ++cases;
      }
    }
  std::printf("WB=%d cases=%ld mismatches=%ld\n", WB, cases, mismatches);
  return mismatches;
}

int main() {
  std::mt19937_64 g(7);
  const long bad = check<1>(g) + check<2>(g) + check<4>(g) + check<8>(g) + check<16>(g);
  return bad == 0 ? 0 : 1;
}
