// Host half of the cuckoo write path (Section 5.3, server steps 1-4).
//
// The placement decision only needs per-slot metadata (which item sits where,
// and each item's two candidate buckets), so it runs on the host; the payload
// never leaves the device.  An insertion yields the final position of every
// item it touched, which is turned into an ordered list of device slot moves:
// copies are ordered so that no slot is overwritten before it has been read,
// and a single temporary slot breaks the rare cycles of a long eviction walk.
//
// Rules (identical on every replica given the same seed and write order):
//   1. at capacity, the oldest item (by first-insert order) is collected and
//      its slot zeroed;
//   2. the item goes to the lowest free slot of b1, else of b2;
//   3. otherwise a bucket e in {b1, b2} is drawn (bit 0 of a draw: 1 -> b2),
//      and up to max_evictions times: a victim slot (draw mod d) of e takes the
//      carried item, the victim becomes the carried item, e becomes the
//      victim's other bucket, and the walk stops at the lowest free slot of e;
//   4. a walk that hits the bound is undone entirely (including step 1) and
//      reported as TPIR_EFULL; the draws it made stay consumed.
// Draws come from splitmix64 (Steele, Lea & Flood 2014) seeded with s_cuckoo.
#include <algorithm>
#include <unordered_map>

#include "tpir_internal.h"

namespace tpir {

namespace {
constexpr uint64_t kNew = ~0ull - 1;  // the item being inserted, before it has a seq
}

CuckooMeta::CuckooMeta(uint64_t n, uint32_t d) : n_(n), d_(d) {
  ring_ = n * d;
  slot_item_.assign(n * d, kEmpty);
  item_slot_.assign(ring_, kEmpty);
  item_b1_.assign(ring_, 0);
  item_b2_.assign(ring_, 0);
}

void CuckooMeta::set_policy(uint64_t capacity, uint32_t max_evictions, uint64_t seed) {
  capacity_ = capacity;
  max_ev_ = max_evictions;
  rng_ = seed;
}

void CuckooMeta::clear() {
  std::fill(slot_item_.begin(), slot_item_.end(), kEmpty);
  std::fill(item_slot_.begin(), item_slot_.end(), kEmpty);
  head_ = next_seq_;
  live_ = 0;
}

uint64_t CuckooMeta::next_rand() {
  rng_ += 0x9E3779B97F4A7C15ull;
  uint64_t x = rng_;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

int64_t CuckooMeta::lowest_free(uint64_t e) const {
  const uint64_t base = e * d_;
  for (uint32_t j = 0; j < d_; ++j)
    if (slot_item_[base + j] == kEmpty) return static_cast<int64_t>(base + j);
  return -1;
}

tpir_status CuckooMeta::insert(uint64_t b1, uint64_t b2, uint64_t payload_idx,
                               std::vector<MoveOp>& ops, uint32_t* evictions, Undo* undo) {
  if (evictions) *evictions = 0;
  if (b1 >= n_ || b2 >= n_) return TPIR_EINVAL;
  const uint64_t rng0 = rng_;

  // undo logs: (slot, previous item) and (item seq, previous slot)
  std::vector<std::pair<uint64_t, uint64_t>> undo_slot, undo_item;
  auto set_slot = [&](uint64_t s, uint64_t item) {
    undo_slot.emplace_back(s, slot_item_[s]);
    slot_item_[s] = item;
  };
  uint64_t new_slot = kEmpty;
  auto place = [&](uint64_t item, uint64_t s) {
    set_slot(s, item);
    if (item == kNew) {
      new_slot = s;
    } else {
      undo_item.emplace_back(item, islot(item));
      islot(item) = s;
    }
  };
  auto cb1 = [&](uint64_t item) { return item == kNew ? b1 : item_b1_[item % ring_]; };
  auto cb2 = [&](uint64_t item) { return item == kNew ? b2 : item_b2_[item % ring_]; };

  const uint64_t old_head = head_, old_live = live_;
  uint64_t gc_slot = kEmpty;
  // step 1: collection of the oldest item
  if (capacity_ > 0 && live_ == capacity_) {
    gc_slot = islot(head_);
    set_slot(gc_slot, kEmpty);
    ++head_;
    --live_;
  }
  // step 2
  int64_t f = lowest_free(b1);
  if (f < 0) f = lowest_free(b2);
  bool placed = false;
  uint32_t moves = 0;
  if (f >= 0) {
    place(kNew, static_cast<uint64_t>(f));
    placed = true;
  } else {
    // step 3
    uint64_t e = (next_rand() & 1u) ? b2 : b1;
    uint64_t carried = kNew;
    for (uint32_t i = 0; i < max_ev_ && !placed; ++i) {
      const uint64_t v = e * d_ + next_rand() % d_;
      const uint64_t victim = slot_item_[v];
      place(carried, v);
      ++moves;
      carried = victim;
      e = (e == cb1(carried)) ? cb2(carried) : cb1(carried);
      const int64_t g = lowest_free(e);
      if (g >= 0) {
        place(carried, static_cast<uint64_t>(g));
        placed = true;
      }
    }
  }
  if (evictions) *evictions = moves;

  if (!placed) {  // step 4: undo everything
    for (auto it = undo_item.rbegin(); it != undo_item.rend(); ++it) islot(it->first) = it->second;
    for (auto it = undo_slot.rbegin(); it != undo_slot.rend(); ++it) slot_item_[it->first] = it->second;
    head_ = old_head;
    live_ = old_live;
    return TPIR_EFULL;
  }

  // commit the new item
  if (undo) {
    undo->head = old_head;
    undo->live = old_live;
    undo->next_seq = next_seq_;
    undo->rng = rng0;
    undo->ring_b1 = item_b1_[next_seq_ % ring_];
    undo->ring_b2 = item_b2_[next_seq_ % ring_];
    undo->ring_slot = item_slot_[next_seq_ % ring_];
  }
  const uint64_t seq = next_seq_++;
  item_b1_[seq % ring_] = b1;
  item_b2_[seq % ring_] = b2;
  islot(seq) = new_slot;
  slot_item_[new_slot] = seq;
  ++live_;

  // ---- device moves: final item of every touched slot vs. original layout
  std::unordered_map<uint64_t, uint64_t> orig_item;  // slot -> item before this insert
  for (const auto& u : undo_slot) orig_item.emplace(u.first, u.second);
  std::unordered_map<uint64_t, uint64_t> orig_slot;  // item -> slot before this insert
  for (const auto& u : undo_item) orig_slot.emplace(u.first, u.second);

  std::vector<std::pair<uint64_t, uint64_t>> copies;  // (dst, src)
  std::vector<uint64_t> touched;
  touched.reserve(orig_item.size());
  for (const auto& kv : orig_item) touched.push_back(kv.first);
  std::sort(touched.begin(), touched.end());
  for (uint64_t s : touched) {
    const uint64_t fin = slot_item_[s];
    if (fin == kEmpty) {
      ops.push_back(MoveOp{s, 0, 2u, 0u});  // collected slot that stays empty
      continue;
    }
    if (fin == seq) continue;  // payload written last
    auto it = orig_slot.find(fin);
    const uint64_t src = (it == orig_slot.end()) ? s : it->second;
    if (src != s) copies.emplace_back(s, src);
  }
  // order the copies: a copy may run once no pending copy still reads its dst
  while (!copies.empty()) {
    bool progressed = false;
    for (size_t i = 0; i < copies.size();) {
      const uint64_t dst = copies[i].first;
      bool needed = false;
      for (size_t j = 0; j < copies.size() && !needed; ++j)
        if (j != i && copies[j].second == dst) needed = true;
      if (!needed) {
        ops.push_back(MoveOp{dst, copies[i].second, 0u, 0u});
        copies.erase(copies.begin() + static_cast<long>(i));
        progressed = true;
      } else {
        ++i;
      }
    }
    if (!progressed) {
      // only cycles are left: park one source in the temporary slot
      const uint64_t s0 = copies[0].second;
      ops.push_back(MoveOp{kTmpSlot, s0, 0u, 0u});
      copies[0].second = kTmpSlot;
    }
  }
  ops.push_back(MoveOp{new_slot, payload_idx, 1u, 0u});
  (void)gc_slot;
  if (undo) {
    undo->slots = std::move(undo_slot);
    undo->items = std::move(undo_item);
  }
  return TPIR_OK;
}

void CuckooMeta::rollback(const Undo& u) {
  // the new item's ring entry, then positions and slots in reverse order
  // (the slot log restores the new item's slot too: it was logged when the
  // item was placed)
  const uint64_t r = u.next_seq % ring_;
  item_b1_[r] = u.ring_b1;
  item_b2_[r] = u.ring_b2;
  item_slot_[r] = u.ring_slot;
  for (auto it = u.items.rbegin(); it != u.items.rend(); ++it) islot(it->first) = it->second;
  for (auto it = u.slots.rbegin(); it != u.slots.rend(); ++it) slot_item_[it->first] = it->second;
  head_ = u.head;
  live_ = u.live;
  next_seq_ = u.next_seq;
  rng_ = u.rng;
}

}  // namespace tpir
