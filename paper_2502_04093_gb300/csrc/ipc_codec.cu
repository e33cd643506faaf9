// Lossless backend of libipcomp (host code): the entropy-coding stage that
// follows predictive coding (Sec. 6.2.1, where the paper runs zstd over the
// plane streams). The GPU container stays the parity contract; this stage
// turns its bytes (or any byte string) into a coded container and back.
//
// Coded container (little-endian):
//   u32 magic "IPCZ", u32 version (2; version 1 is still read), u64 raw
//   length, u32 log2 of the block size, u32 block count, then one u32 per
//   block (its record's bytes), then the block records. A block is the next
//   2^log2 raw bytes (the last one shorter). Record: u8 mode; mode 0 holds
//   the raw bytes; modes 1 and 2 hold 256 u16 symbol frequencies (summing to
//   4096) and an order-0 rANS byte stream (range asymmetric numeral
//   systems, Duda 2013; 32-bit states kept in [2^23, 2^31), byte-wise
//   renormalisation). Mode 1 (written by version 1) has one state, whose
//   final value leads the stream. Mode 2 (written now) has two states that
//   take the symbols in turn -- symbol i uses state i mod 2 -- and share the
//   byte stream (interleaved rANS, Giesen 2014): the stream leads with the
//   final values of states 0 and 1, and each symbol's renormalisation bytes
//   follow in symbol order. Two states let the decoder work on two
//   independent dependency chains.
// Frequencies: f_s = 0 for absent bytes, else max(1, floor(c_s 4096 / n));
// the difference to 4096 is then settled one unit at a time on the symbol
// of largest frequency (lowest byte value on ties; never below 1). A block
// is stored (mode 0) when its coded record would not be smaller.
// Blocks are independent: both directions run them on host threads.
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "ipc.h"
#include "ipc_internal.h"

namespace {

constexpr uint32_t kMagicZ = 0x5A435049u;  // "IPCZ"
constexpr uint32_t kVersionZ = 2;  // written; 1 and 2 are read
constexpr int kScale = 12;
constexpr uint32_t kTotal = 1u << kScale;
constexpr uint32_t kLow = 1u << 23;  // lower end of the normalised state interval
constexpr uint64_t kHead = 24;       // fixed header bytes
constexpr uint64_t kTable = 512;     // frequency table bytes

int err(int code, const char* what) {
  ipc::set_last_error(what);
  return code;
}

void put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
void put64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

void normalise(const uint8_t* src, uint64_t n, uint32_t f[256]) {
  // four interleaved counter tables: runs of one byte value do not chain
  // every increment on the same counter
  uint64_t c4[4][256] = {};
  uint64_t i = 0;
  for (; i + 4 <= n; i += 4) {
    ++c4[0][src[i]];
    ++c4[1][src[i + 1]];
    ++c4[2][src[i + 2]];
    ++c4[3][src[i + 3]];
  }
  for (; i < n; ++i) ++c4[0][src[i]];
  uint64_t c[256];
  for (int s = 0; s < 256; ++s) c[s] = c4[0][s] + c4[1][s] + c4[2][s] + c4[3][s];
  int64_t sum = 0;
  for (int s = 0; s < 256; ++s) {
    f[s] = c[s] == 0 ? 0 : (uint32_t)std::max<uint64_t>(1, c[s] * kTotal / n);
    sum += f[s];
  }
  auto largest = [&](bool above_one) {
    int m = -1;
    for (int s = 0; s < 256; ++s)
      if ((!above_one || f[s] > 1) && (m < 0 || f[s] > f[m])) m = s;
    return m;
  };
  while (sum < (int64_t)kTotal) {
    ++f[largest(false)];
    ++sum;
  }
  while (sum > (int64_t)kTotal) {
    --f[largest(true)];
    --sum;
  }
}

// Division of a state x < 2^31 by a frequency 1 <= f <= 4096 as a multiply
// and shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 f) and m = ceil(2^(31+l) / f),
// floor(x / f) = floor(x m / 2^(31+l)) for every x < 2^31, and x m < 2^64.
struct Recip {
  uint64_t m;
  uint32_t shift;
};
Recip recip(uint32_t f) {
  uint32_t l = 0;
  while ((1u << l) < f) ++l;
  const uint64_t num = uint64_t(1) << (31 + l);
  return Recip{(num + f - 1) / f, 31 + l};
}

// Codes one block of n bytes into `rec` (capacity 1 + n: a record is never
// larger than the stored form); returns the record's size.
uint64_t encode_block(const uint8_t* src, uint64_t n, uint8_t* rec, std::vector<uint8_t>* tmp) {
  uint32_t f[256], start[256], xmax[256];
  Recip rc[256];
  normalise(src, n, f);
  uint32_t acc = 0;
  for (int s = 0; s < 256; ++s) {
    start[s] = acc;
    acc += f[s];
    xmax[s] = ((kLow >> kScale) << 8) * f[s];
    rc[s] = f[s] ? recip(f[s]) : Recip{0, 0};
  }
  // the rANS bytes are written backwards from the end of a scratch buffer:
  // at most 2 bytes per symbol (a frequency >= 1 of 4096 adds at most 12
  // bits of state) plus the two final states
  tmp->resize(2 * n + 12);
  uint8_t* const end = tmp->data() + tmp->size();
  uint8_t* p = end;
  uint32_t xs[2] = {kLow, kLow};
  for (uint64_t i = n; i-- > 0;) {
    const uint32_t s = src[i];
    uint32_t& x = xs[i & 1];
    // shift out low bytes while x >= xmax_s: with x < 2^31 and
    // xmax_s >= 2^19 that is at most two, decided without a branch (the
    // count is data-dependent); both candidate bytes are stored, p moves by
    // the count (the space below p is unused so far: p >= end - 2 i)
    const uint32_t nb = (uint32_t)(x >= xmax[s]) + (uint32_t)((uint64_t)x >= ((uint64_t)xmax[s] << 8));
    p[-1] = (uint8_t)(x & 0xFF);
    p[-2] = (uint8_t)((x >> 8) & 0xFF);
    p -= nb;
    x >>= 8 * nb;
    // x < 2^31 here (x < xmax <= 2^31); q = floor(x / f_s)
    const uint32_t q = (uint32_t)(((uint64_t)x * rc[s].m) >> rc[s].shift);
    x = (q << kScale) + (x - q * f[s]) + start[s];
  }
  p -= 4;
  put32(p, xs[1]);
  p -= 4;
  put32(p, xs[0]);
  const uint64_t coded = (uint64_t)(end - p);
  if (1 + kTable + coded >= 1 + n) {  // no gain: stored
    rec[0] = 0;
    std::memcpy(rec + 1, src, n);
    return 1 + n;
  }
  rec[0] = 2;
  for (int s = 0; s < 256; ++s) {
    rec[1 + 2 * s] = (uint8_t)(f[s] & 0xFF);
    rec[2 + 2 * s] = (uint8_t)(f[s] >> 8);
  }
  std::memcpy(rec + 1 + kTable, p, coded);
  return 1 + kTable + coded;
}

// Decodes one record into n bytes; false when it is not a valid coding of n
// bytes. The slot table holds, per slot of [0, 4096), its symbol, the
// symbol's frequency and the slot's offset in the symbol's range, so that a
// step is one table load.
bool decode_block(const uint8_t* rec, uint64_t len, uint8_t* dst, uint64_t n,
                  std::vector<uint32_t>* slots) {
  if (len < 1) return false;
  if (rec[0] == 0) {
    if (len != 1 + n) return false;
    std::memcpy(dst, rec + 1, n);
    return true;
  }
  const int nstates = rec[0];
  if ((nstates != 1 && nstates != 2) || len < 1 + kTable + 4 * (uint64_t)nstates) return false;
  uint32_t f[256], acc = 0;
  for (int s = 0; s < 256; ++s) {
    f[s] = (uint32_t)rec[1 + 2 * s] | ((uint32_t)rec[2 + 2 * s] << 8);
    acc += f[s];
  }
  if (acc != kTotal) return false;
  slots->resize(kTotal);
  uint32_t* const tab = slots->data();
  // entry: symbol (bits 0-7), frequency - 1 (bits 8-19), offset in the
  // symbol's range (bits 20-31)
  for (uint32_t s = 0, slot = 0; s < 256; ++s)
    for (uint32_t k = 0; k < f[s]; ++k, ++slot) tab[slot] = s | ((f[s] - 1) << 8) | (k << 20);
  const uint8_t* p = rec + 1 + kTable;
  const uint8_t* const end = rec + len;
  uint32_t xs[2] = {get32(p), nstates == 2 ? get32(p + 4) : kLow};
  p += 4 * nstates;
  bool ok = true;
  // one symbol from state x, then its renormalisation: x >= f (2^23 >> 12)
  // >= 2^11 after the step, so at most two bytes bring it back to
  // [2^23, 2^31); the count is taken without a branch while two bytes are
  // left to read, byte by byte near the end of the stream
  auto step = [&](uint32_t& x, uint8_t* out) {
    const uint32_t e = tab[x & (kTotal - 1)];
    *out = (uint8_t)e;
    x = (((e >> 8) & 0xFFF) + 1) * (x >> kScale) + (e >> 20);
    if (end - p >= 2) {
      const uint32_t nb = (uint32_t)(x < kLow) + (uint32_t)(x < (kLow >> 8));
      const uint32_t two = ((uint32_t)p[0] << 8) | p[1];
      x = (x << (8 * nb)) | (two >> (8 * (2 - nb)));
      p += nb;
    } else {
      while (x < kLow) {
        if (p >= end) {
          ok = false;
          x = kLow;  // ends the loop; the record is refused
          break;
        }
        x = (x << 8) | *p++;
      }
    }
  };
  if (nstates == 1) {
    for (uint64_t i = 0; i < n && ok; ++i) step(xs[0], dst + i);
  } else {
    uint64_t i = 0;
    for (; i + 1 < n && ok; i += 2) {
      step(xs[0], dst + i);
      step(xs[1], dst + i + 1);
    }
    if (i < n && ok) step(xs[0], dst + i);
  }
  // the encoder started every state from kLow and used every byte
  return ok && p == end && xs[0] == kLow && xs[1] == kLow;
}

int threads_for(int nthreads, uint64_t nblocks) {
  unsigned t = nthreads > 0 ? (unsigned)nthreads : std::max(1u, std::thread::hardware_concurrency());
  t = std::min<unsigned>(t, 16);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(t, nblocks));
}

// Runs body(i) for i in [0, n) on up to `nt` threads.
template <class F>
void parallel_blocks(uint64_t n, int nt, F body) {
  std::atomic<uint64_t> next{0};
  auto run = [&]() {
    for (uint64_t i; (i = next.fetch_add(1)) < n;) body(i);
  };
  std::vector<std::thread> th;
  for (int k = 1; k < nt; ++k) {
    try {
      th.emplace_back(run);
    } catch (...) {
      break;  // the others share the work
    }
  }
  run();
  for (auto& t : th) t.join();
}

}  // namespace

extern "C" {

int ipc_encode_container(const void* raw, uint64_t raw_len, int block_log2, void* out,
                         uint64_t* out_len, int nthreads) {
  ipc::set_last_error("");
  if (!out_len || (!raw && raw_len)) return err(IPC_EINVAL, "null argument");
  if (block_log2 == 0) block_log2 = 20;
  if (block_log2 < 12 || block_log2 > 26) return err(IPC_EINVAL, "block size");
  const uint64_t bs = uint64_t(1) << block_log2;
  const uint64_t nb = (raw_len + bs - 1) / bs;
  if (nb > 0xFFFFFFFFull) return err(IPC_EINVAL, "too many blocks");
  const uint64_t bound = kHead + 4 * nb + nb + raw_len;
  if (!out) {
    *out_len = bound;
    return IPC_OK;
  }
  const uint8_t* src = (const uint8_t*)raw;
  // every block is coded into its own slot of a bound-sized scratch, then
  // the records are packed behind the table of their sizes
  std::vector<uint8_t> slots(nb + raw_len);
  std::vector<uint64_t> size(nb), slot_off(nb);
  for (uint64_t i = 0; i < nb; ++i) slot_off[i] = i * (bs + 1);
  parallel_blocks(nb, threads_for(nthreads, nb), [&](uint64_t i) {
    thread_local std::vector<uint8_t> tmp;
    const uint64_t n = std::min(bs, raw_len - i * bs);
    size[i] = encode_block(src + i * bs, n, slots.data() + slot_off[i], &tmp);
  });
  uint64_t total = kHead + 4 * nb;
  for (uint64_t i = 0; i < nb; ++i) total += size[i];
  if (*out_len < total) return err(IPC_EINVAL, "output capacity too small");
  uint8_t* o = (uint8_t*)out;
  put32(o, kMagicZ);
  put32(o + 4, kVersionZ);
  put64(o + 8, raw_len);
  put32(o + 16, (uint32_t)block_log2);
  put32(o + 20, (uint32_t)nb);
  uint64_t pos = kHead + 4 * nb;
  for (uint64_t i = 0; i < nb; ++i) {
    put32(o + kHead + 4 * i, (uint32_t)size[i]);
    std::memcpy(o + pos, slots.data() + slot_off[i], size[i]);
    pos += size[i];
  }
  *out_len = total;
  return IPC_OK;
}

int ipc_decode_container(const void* coded, uint64_t coded_len, void* out, uint64_t* out_len,
                         int nthreads) {
  ipc::set_last_error("");
  if (!coded || !out_len) return err(IPC_EINVAL, "null argument");
  const uint8_t* c = (const uint8_t*)coded;
  if (coded_len < kHead || get32(c) != kMagicZ || (get32(c + 4) != 1 && get32(c + 4) != 2))
    return err(IPC_ECORRUPT, "not a coded container");
  const uint64_t raw_len = get64(c + 8);
  const uint32_t lg = get32(c + 16);
  const uint64_t nb = get32(c + 20);
  if (lg < 12 || lg > 26) return err(IPC_ECORRUPT, "block size");
  const uint64_t bs = uint64_t(1) << lg;
  if (nb != (raw_len + bs - 1) / bs || kHead + 4 * nb > coded_len)
    return err(IPC_ECORRUPT, "block count");
  if (!out) {
    *out_len = raw_len;
    return IPC_OK;
  }
  if (*out_len < raw_len) return err(IPC_EINVAL, "output capacity too small");
  std::vector<uint64_t> off(nb + 1);
  off[0] = kHead + 4 * nb;
  for (uint64_t i = 0; i < nb; ++i) off[i + 1] = off[i] + get32(c + kHead + 4 * i);
  if (off[nb] != coded_len) return err(IPC_ECORRUPT, "block sizes");
  std::atomic<int> bad{0};
  uint8_t* o = (uint8_t*)out;
  parallel_blocks(nb, threads_for(nthreads, nb), [&](uint64_t i) {
    thread_local std::vector<uint32_t> slots;
    const uint64_t n = std::min(bs, raw_len - i * bs);
    if (!decode_block(c + off[i], off[i + 1] - off[i], o + i * bs, n, &slots)) bad.store(1);
  });
  if (bad.load()) return err(IPC_ECORRUPT, "a block does not decode to its length");
  *out_len = raw_len;
  return IPC_OK;
}

}  // extern "C"
