// Host-only: the key under which the multi-solve engine caches the CUDA graph of a tick.
//
// A tick's graph bakes in the device pointers of every active solve and the pinned host
// mirrors its status copies write into.  It may be replayed only for exactly the same solves
// in exactly the same units.  A solve is named by its submission number, which the engine
// hands out once per cmcg_engine_submit and never reuses: a handle address or a slot index
// is not enough, because a finished solve's handle can be destroyed and a new one created at
// the same address and admitted into the same slot.
//
// No CUDA types here, so that the rules can be checked on a host without a GPU.
#pragma once
#include <cstddef>
#include <vector>

namespace cmcg {
namespace detail {

class TickSignature {
 public:
    void clear() { v_.clear(); }
    bool empty() const { return v_.empty(); }
    // One active slot: its index, its unit of work this tick, and its submission number.
    void add(int slot, int unit, long long submission) {
        v_.push_back(slot);
        v_.push_back(unit);
        v_.push_back(submission);
    }
    bool operator==(const TickSignature& o) const { return v_ == o.v_; }
    bool operator!=(const TickSignature& o) const { return v_ != o.v_; }
    // Does the signature include this slot (any unit, any submission)?
    bool names_slot(int slot) const {
        for (size_t i = 0; i < v_.size(); i += 3)
            if (v_[i] == slot) return true;
        return false;
    }

 private:
    std::vector<long long> v_;
};

}  // namespace detail
}  // namespace cmcg
