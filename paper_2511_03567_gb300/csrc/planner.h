// Runtime planner interface (planner.cu).
#pragma once
#include <map>
#include <string>
#include <vector>

#include "internal.h"

class Planner {
 public:
  Planner(const Dims& d, const TensorView* tensors, const TensorView* outs, const double* ones);
  // Plan one term into `prog`; false if the term does not fit the views.
  bool add_term(const RicTermDesc& t, Program* prog);
  // Elements of the intermediate arena the planned programs need.
  int64_t arena_size() const { return arena_size_; }
  int64_t cse_hits() const { return cse_hits_; }
  // Patch arena offsets of `prog` (planned by this planner) into addresses.
  void finalize(Program* prog, double* arena);
  // One contraction C[...] += alpha * A[...] B[...] between explicit operands.
  void emit(const Operand& A, const Operand& B, const Operand& C, const int64_t* ext, double alpha,
            int arena_flags, Program* prog);

 private:
  bool make_operand(const TensorView& tv, int tensor_tag, int nidx, const uint8_t* idx,
                    const uint8_t* mask, Operand* op);
  Operand intermediate(const Operand& A, const Operand& B, const std::vector<int>& keep,
                       const int64_t* ext, Program* prog);

  Dims d_;
  TensorView tensors_[NTENSOR];
  TensorView outs_[NOUT];
  const double* ones_;
  std::map<std::string, int64_t> cse_;
  int64_t arena_size_ = 0;
  int64_t cse_hits_ = 0;
  std::map<int64_t, int> producer_level_;  // arena offset -> level of its producing op
};
