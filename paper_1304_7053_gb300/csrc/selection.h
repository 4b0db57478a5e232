// Kernel-variant selection for the fixed-size entry points.
//
// The paper's kernels take a launch configuration that is "tunable for minor
// gains" and suggests more specialised kernels per size (Section 6).  Here a
// problem class (type, m, n, k, opA transposed, opB transposed, beta == 0,
// batch-size class) is mapped to one of the library's kernel variants, from,
// in order: the selection table (measured choices, e.g. from the autotuner),
// the cost model's predicted choice (a perceptron evaluated once per class
// with this library's own kernels), and the built-in default rule.
#pragma once

namespace sbg {

// floor(log10(batch)) clamped to 0..7
int size_class(int batch);
// number of public variants of a (type, m, n, k) problem; 0 when invalid
int variants_for(int type, int m, int n, int k);
// the built-in choice without a table entry or cost model
int default_variant(int type, int m, int n, int k, int beta_zero, int sc);
// the choice under the current selector mode
int select_variant(int type, int m, int n, int k, int ta, int tb, int beta_zero, int sc);
// remember the variant the calling thread's latest fixed-size call used
void note_variant(int v);

}  // namespace sbg
