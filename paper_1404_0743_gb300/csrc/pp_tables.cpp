// pp_tables.cpp -- host construction of the library's constant tables.
//
// Quadrant codes, rotation-minimal quadrant lists and the standardisation
// map follow the paper's Section "Data layout and distribution": a section
// is a 4-D array whose axis q runs over the quadrant-q patterns that are
// least among their four rotations.  The rotated five-in-a-row forms follow
// "Abstracting over rotations" (sets of quadrant turns that complete a line).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "pp_internal.h"

namespace pp {
namespace {

int pow3i(int e) {
  int p = 1;
  while (e-- > 0) p *= 3;
  return p;
}

// One anticlockwise quarter turn of a ternary quadrant code: the stone at
// local (r, c) moves to (2 - c, r).
int rotate_code(int code) {
  int digit[9], out = 0;
  for (int i = 0; i < 9; i++, code /= 3) digit[i] = code % 3;
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) out += digit[3 * r + c] * pow3i(3 * (2 - c) + r);
  return out;
}

// The local action of board symmetry s on a quadrant's pattern: a mirror
// (r, c) -> (r, 2 - c) when s >= 4, then s & 3 anticlockwise turns.
int symmetry_code(int s, int code) {
  if (s >> 2) {
    int digit[9], out = 0;
    for (int i = 0; i < 9; i++, code /= 3) digit[i] = code % 3;
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) out += digit[3 * r + c] * pow3i(3 * r + 2 - c);
    code = out;
  }
  for (int k = 0; k < (s & 3); k++) code = rotate_code(code);
  return code;
}

struct LineInfo {
  uint32_t part[4];  // 9-bit local cells of the line in quadrant q (0 if none)
  int quads;         // bit mask of touched quadrants
};

std::vector<LineInfo> all_lines() {
  std::vector<LineInfo> out;
  const int dir[4][2] = {{0, 1}, {1, 0}, {1, 1}, {1, -1}};
  for (int R = 0; R < 6; R++)
    for (int C = 0; C < 6; C++)
      for (auto& d : dir) {
        int R4 = R + 4 * d[0], C4 = C + 4 * d[1];
        if (R4 < 0 || R4 > 5 || C4 < 0 || C4 > 5) continue;
        LineInfo l{};
        for (int i = 0; i < 5; i++) {
          int r = R + i * d[0], c = C + i * d[1];
          int q = 2 * (r >= 3) + (c >= 3);
          l.part[q] |= 1u << (3 * (r % 3) + c % 3);
          l.quads |= 1 << q;
        }
        out.push_back(l);
      }
  return out;
}

// S_{l,q}(x): turns t with l's quadrant-q cells inside rot^t(x).
uint32_t cover_set(uint32_t part, uint32_t x) {
  uint32_t s = 0, y = x;
  for (int t = 0; t < 4; t++, y = rotate9(y))
    if ((y & part) == part) s |= 1u << t;
  return s;
}

uint32_t rep_form(uint32_t s) { return s * 0x1111u; }
uint32_t e_form(uint32_t s) {
  uint32_t e = 0;
  for (int j = 0; j < 4; j++)
    if (s >> j & 1) e |= 0xFu << (4 * j);
  return e;
}

void put16(uint32_t* w, int slot_word, int line, uint32_t form) {
  w[slot_word + line / 2] |= form << (16 * (line % 2));
}

void build(HostTables& t) {
  std::memset(&t, 0, sizeof(t));
  // quadrant decode
  for (int code = 0; code < kQStates; code++) {
    uint32_t b = 0, w = 0;
    int x = code;
    for (int i = 0; i < 9; i++, x /= 3) {
      if (x % 3 == 1) b |= 1u << i;
      if (x % 3 == 2) w |= 1u << i;
    }
    t.qdecode[code] = b | w << 9 | (uint32_t)__builtin_popcount(b) << 18 |
                      (uint32_t)__builtin_popcount(w) << 22;
  }
  // rotation-minimal lists grouped by counts
  std::vector<int> minimal[10][10];
  for (int code = 0; code < kQStates; code++) {
    int r1 = rotate_code(code), r2 = rotate_code(r1), r3 = rotate_code(r2);
    if (code <= r1 && code <= r2 && code <= r3) {
      uint32_t d = t.qdecode[code];
      minimal[(d >> 18) & 15][(d >> 22) & 15].push_back(code);
    }
  }
  int off = 0;
  for (int b = 0; b < 10; b++)
    for (int w = 0; w < 10; w++) {
      t.qoff[b][w] = off;
      t.qdim[b][w] = (int)minimal[b][w].size();
      for (int code : minimal[b][w]) t.qlist[off++] = (uint16_t)code;
    }
  // standardisation: y = rot^u(m), m the least of y's rotations; the
  // smallest s with rot^s(y) = m gives u = (4 - s) mod 4
  for (int code = 0; code < kQStates; code++) {
    int y = code, best = code, best_s = 0;
    for (int s = 1; s < 4; s++) {
      y = rotate_code(y);
      if (y < best) best = y, best_s = s;
    }
    uint32_t d = t.qdecode[best];
    auto& lst = minimal[(d >> 18) & 15][(d >> 22) & 15];
    int rank = (int)(std::lower_bound(lst.begin(), lst.end(), best) - lst.begin());
    t.standard[code] = (uint32_t)rank | (uint32_t)((4 - best_s) & 3) << 16;
  }
  // one-move table: patterns and, for one-empty-cell states, the child
  for (int i = 0; i < kMinStates; i++) {
    const int code = t.qlist[i];
    const uint32_t d = t.qdecode[code], b = d & 0x1FF, w = (d >> 9) & 0x1FF;
    const uint32_t empty = ~(b | w) & 0x1FFu;
    for (int c = 1; c <= 2; c++) {
      t.qline[c - 1][i][0] = b | w << 9;
      t.qline[c - 1][i][1] = 0;
      if (__builtin_popcount(empty) == 1) {
        const int e = __builtin_ctz(empty);
        const uint32_t s = t.standard[code + c * pow3i(e)];
        t.qline[c - 1][i][1] = (uint32_t)e | (s & 0xFFFFu) << 4 | (s >> 16) << 13;
      }
    }
  }
  for (int c = 0; c < 2; c++)
    for (int b = 0; b < 10; b++)
      for (int w = 0; b + w <= 9; w++) {
        const int o = t.qoff[b][w], n = t.qdim[b][w];
        std::vector<int> pos(n);
        for (int p = 0; p < n; p++) pos[p] = p;
        auto key = [&](int p) {  // child rank j, then turn u
          const uint32_t y = t.qline[c][o + p][1];
          return ((y >> 4) & 0x1FFu) << 2 | ((y >> 13) & 3u);
        };
        std::stable_sort(pos.begin(), pos.end(), [&](int a, int z) { return key(a) < key(z); });
        for (int k = 0; k < n; k++) {
          const uint32_t y = t.qline[c][o + pos[k]][1];
          t.qsorted[c][o + k][0] = t.qline[c][o + pos[k]][0];
          t.qsorted[c][o + k][1] = y | (uint32_t)pos[k] << 16;
          t.qsorted[c][o + k][2] = 0;
          t.qsorted[c][o + k][3] = 0;
          if (b + w == 8) {  // one empty cell: the child's minimal pattern
            const int cb = b + (c == 0), cw = w + (c == 1);
            const uint32_t code = t.qlist[t.qoff[cb][cw] + ((y >> 4) & 0x1FFu)];
            t.qsorted[c][o + k][2] = t.qdecode[code] & 0x3FFFFu;
          }
        }
      }
  // symmetry images of the minimal states (same counts, so the rank is
  // within the same list)
  for (int sy = 0; sy < 8; sy++)
    for (int i = 0; i < kMinStates; i++) {
      const uint32_t st = t.standard[symmetry_code(sy, t.qlist[i])];
      t.dmin[sy][i] = (uint16_t)((st & 0xFFFu) | (st >> 16) << 12);
    }
  // subsets of the midgame slots with at most c of them, c = 0..8
  {
    int at = 0;
    for (int c = 0; c <= kMaxEmpty / 2; c++)
      for (uint32_t v = 0; v < (1u << kMaxEmpty); v++)
        if (__builtin_popcount(v) <= c) t.subsets[at++] = (uint16_t)v;
    if (at != kCappedSubsets) std::abort();
  }
  // five-in-a-row forms
  std::vector<LineInfo> lines = all_lines();
  auto group = [&](int quads) {
    std::vector<LineInfo> g;
    for (auto& l : lines)
      if (l.quads == quads) g.push_back(l);
    return g;
  };
  struct Pair { int a, b, slot_a, slot_b; };  // a = rep quadrant, b = E quadrant
  // slot word offsets: A = 0, B = 3, C = 6
  const Pair pairs[6] = {
      {0, 1, 0, 0},  // P01: q0.A & q1.A
      {0, 2, 3, 3},  // P02: q0.B & q2.B
      {0, 3, 6, 6},  // P03: q0.C & q3.C
      {2, 1, 6, 6},  // P12: q2.C & q1.C
      {3, 1, 3, 3},  // P13: q3.B & q1.B
      {2, 3, 0, 0},  // P23: q2.A & q3.A
  };
  struct Triple { int quads, a, b, gate; };
  const Triple triples[4] = {
      {0b1011, 0, 1, 3},  // T0
      {0b1101, 0, 2, 3},  // T1
      {0b0111, 0, 1, 2},  // T2
      {0b1110, 2, 1, 3},  // T3
  };
  for (uint32_t x = 0; x < 512; x++) {
    for (const Pair& p : pairs) {
      auto g = group(1 << p.a | 1 << p.b);
      for (size_t j = 0; j < g.size(); j++) {
        put16(t.forms[p.a][x], p.slot_a, (int)j, rep_form(cover_set(g[j].part[p.a], x)));
        put16(t.forms[p.b][x], p.slot_b, (int)j, e_form(cover_set(g[j].part[p.b], x)));
      }
    }
    for (int ti = 0; ti < 4; ti++) {
      const Triple& tr = triples[ti];
      auto g = group(tr.quads);
      const LineInfo& l = g.at(0);
      put16(t.forms[tr.a][x], 7, ti, rep_form(cover_set(l.part[tr.a], x)));
      put16(t.forms[tr.b][x], 7, ti, e_form(cover_set(l.part[tr.b], x)));
      t.forms[tr.gate][x][9] |= cover_set(l.part[tr.gate], x) << (4 * ti);
    }
  }
}

}  // namespace

int symmetry_pattern(int s, int code) { return symmetry_code(s, code); }

uint32_t rotate9(uint32_t mask) {
  uint32_t out = 0;
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++)
      if (mask >> (3 * r + c) & 1) out |= 1u << (3 * (2 - c) + r);
  return out;
}

const HostTables& host_tables() {
  static HostTables* t = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    t = new HostTables;
    build(*t);
  });
  return *t;
}

std::vector<pp_section_desc> slice_sections(int n, uint64_t* total) {
  const HostTables& t = host_tables();
  std::vector<pp_section_desc> out;
  const int B = (n + 1) / 2, W = n / 2;
  std::vector<std::array<int, 2>> qc;
  for (int b = 0; b < 10; b++)
    for (int w = 0; b + w <= 9; w++) qc.push_back({b, w});
  uint64_t offset = 0;
  for (auto& a : qc)
    for (auto& b : qc)
      for (auto& c : qc) {
        int b3 = B - a[0] - b[0] - c[0], w3 = W - a[1] - b[1] - c[1];
        if (b3 < 0 || w3 < 0 || b3 + w3 > 9) continue;
        pp_section_desc d{};
        const int bw[4][2] = {{a[0], a[1]}, {b[0], b[1]}, {c[0], c[1]}, {b3, w3}};
        uint64_t size = 1;
        for (int q = 0; q < 4; q++) {
          d.bw[q][0] = (uint8_t)bw[q][0];
          d.bw[q][1] = (uint8_t)bw[q][1];
          d.dim[q] = (uint16_t)t.qdim[bw[q][0]][bw[q][1]];
          size *= d.dim[q];
        }
        d.offset = offset;
        offset += size;
        out.push_back(d);
      }
  if (total) *total = offset;
  return out;
}

int least_image(const uint8_t bw[4][2], uint8_t out[4][2]) {
  int best_s = -1;
  for (int sy = 0; sy < 8; sy++) {
    uint8_t img[4][2];
    for (int q = 0; q < 4; q++) {
      img[sym_qmap(sy, q)][0] = bw[q][0];
      img[sym_qmap(sy, q)][1] = bw[q][1];
    }
    if (best_s < 0 || std::memcmp(img, out, sizeof img) < 0) {
      std::memcpy(out, img, sizeof img);
      best_s = sy;
    }
  }
  return best_s;
}

std::vector<pp_section_desc> slice_sections_d4(int n, uint64_t* total) {
  std::vector<pp_section_desc> out;
  uint64_t offset = 0;
  for (pp_section_desc d : slice_sections(n, nullptr)) {
    uint8_t least[4][2];
    least_image(d.bw, least);
    if (std::memcmp(least, d.bw, sizeof least) != 0) continue;
    d.offset = offset;
    offset += (uint64_t)d.dim[0] * d.dim[1] * d.dim[2] * d.dim[3];
    out.push_back(d);
  }
  if (total) *total = offset;
  return out;
}

int section_index(const std::vector<pp_section_desc>& secs, const uint8_t bw[4][2]) {
  auto key = [](const uint8_t x[4][2]) {
    uint64_t k = 0;
    for (int q = 0; q < 4; q++) k = k * 100 + x[q][0] * 10 + x[q][1];
    return k;
  };
  uint64_t want = key(bw);
  size_t lo = 0, hi = secs.size();
  while (lo < hi) {  // sections are in increasing key order
    size_t mid = (lo + hi) / 2;
    uint64_t k = key(secs[mid].bw);
    if (k == want) return (int)mid;
    if (k < want)
      lo = mid + 1;
    else
      hi = mid;
  }
  return -1;
}

}  // namespace pp
