// Internal: definitions of the C-ABI handles and the error guard shared by
// the translation units that implement include/symtensor.h.
#pragma once

#include <memory>
#include <new>
#include <string>

#include "../../include/symtensor.h"
#include "plan.h"
#include "structure.h"

struct sym_tensor_s {
  sym::Tensor t;
};
struct sym_plan_s {
  std::unique_ptr<sym::Plan> p;
};

namespace sym {

// thread-local message of the last failed call (sym_last_error)
std::string& last_error();

// Run f, turning exceptions into error codes and messages.
template <class F>
int guard(F&& f) {
  try {
    last_error().clear();
    return f();
  } catch (const Error& e) {
    last_error() = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    last_error() = "host allocation failed";
    return SYM_ERR_OOM;
  } catch (const std::exception& e) {
    last_error() = e.what();
    return SYM_ERR_ARG;
  }
}

// Result structure of contracting A and B (legs, total charge, tree).
Tensor contraction_result(const Tensor& a, const Tensor& b, const std::vector<int>& pa, const std::vector<int>& pb,
                          const int* tree_c);

}  // namespace sym
