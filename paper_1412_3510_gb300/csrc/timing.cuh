// Stage timing hooks (see timing.cu).
#pragma once

#include "internal.cuh"

namespace rpca {

enum TimedKind {
    kTimeApply = 0, kTimeAdjoint = 1, kTimeRenorm = 2, kTimeSmallSvd = 3, kTimeResid = 4,
    kTimeGram = 5, kTimeChol = 6, kTimeTrsm = 7, kTimeCentre = 8, kTimeLift = 9,
    kTimeApplyKernel = 10, kTimeAdjointKernel = 11     // the pass kernel alone (no operand split)
};

bool timing_on();

class TimedScope {
  public:
    TimedScope(int kind, cudaStream_t s);
    ~TimedScope();
    TimedScope(const TimedScope &) = delete;
    TimedScope &operator=(const TimedScope &) = delete;

  private:
    int kind_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace rpca
