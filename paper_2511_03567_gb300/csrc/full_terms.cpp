// Unfiltered BCH-2 ("FULL") spin-free term tables: every term of
// H + [H,T] + 1/2[[H,T],T] without the RIC neglect rules of Sec. 2.2
// (cumulants up to lambda_3).  The generated table is committed gzipped
// (csrc/ric_terms_full.inc.gz, written by gen/emit.py --full); the build
// unpacks it next to the objects and compiles this host-only unit.
#include <stddef.h>

#include "internal.h"
#include "ric_terms_full.inc"

const RicTermDesc* ric_full_terms(int which, size_t* count) {
  if (which == 0) {
    *count = sizeof(kFullResidualTerms) / sizeof(kFullResidualTerms[0]);
    return kFullResidualTerms;
  }
  *count = sizeof(kFullEnergyTerms) / sizeof(kFullEnergyTerms[0]);
  return kFullEnergyTerms;
}
