// Host-side program handling: validation and typing, canonical renumbering,
// lookup of a compile-time instantiation, and lowering to register code for
// the generic interpreter.  Pure host C++ (no CUDA calls), so every check
// runs without a GPU.
#pragma once

#include <stdint.h>

#include <string>

#include "../../include/salt.h"
#include "interp.cuh"
#include "shapes.h"

namespace salt {

struct Analysis {
  int nred = 0;
  int max_depth = 0;
  uint32_t used_vecs = 0;   // user operand indices referenced
  uint32_t stored_vecs = 0; // user operand indices stored
  uint32_t used_scals = 0;
  uint32_t used_dscals = 0; // device scalar indices referenced
  bool scalar_nodes = false; // DSCAL or a scalar-typed operation present
};

// Validates `prog` against nvecs / nscal / ndscal.  On failure fills `err`.
// ADD, SUB, MUL and DIV take two vectors or two scalars, NEG a vector or a
// scalar; SMUL a scalar below a vector.
salt_status analyse(const salt_insn* prog, int nprog, int nvecs, int nscal, Analysis* out,
                    std::string* err, int ndscal = 0);

struct Canonical {
  int len = 0;
  int code[kMaxProg];          // pack(op, canonical arg)
  int nvec = 0, nscal = 0;     // canonical operand counts
  int vec_user[kMaxVecs];      // canonical vector slot -> user index
  int scal_user[kMaxScals];    // canonical scalar slot -> user index
  uint32_t load_mask = 0;      // canonical slots read before written
  uint32_t store_mask = 0;     // canonical slots stored
  int nred = 0;
};

// Renumbers operands in order of first appearance (call after analyse()).
void canonicalise(const salt_insn* prog, int nprog, Canonical* c);

// Shape id of a canonical program, or -1 if it has no instantiation.
int find_shape(const Canonical& c);

// Lowers a canonical program to interpreter register code.  Returns false if
// the register code would exceed kMaxRegCode instructions.
bool lower(const Canonical& c, RegInsn* code, int* len);

// A program with its scalar subexpressions hoisted (Section 4.2: values
// that do not depend on the element are computed once, by init /
// load_once).  Every maximal scalar subtree other than a bare SCAL -- a
// scalar operation, or a DSCAL -- is removed and one SCAL of a new slot
// (numbered from the user's nscal up) takes the place of its root; equal
// subtrees share a slot.
struct Hoisted {
  salt_insn prog[kMaxProg];
  int nprog = 0;
  int nscal = 0;               // user scalars + hoisted slots
  int nhoist = 0;
  uint32_t mask[kMaxScals] = {};  // tokens (bit pc of the original program)
                                  // of subexpression j, in postfix order
  bool device = false;         // some subexpression reads a DSCAL
};

// Call after analyse() succeeded.  SALT_ERR_PROGRAM if the slots exceed
// kMaxScals.
salt_status hoist_scalars(const salt_insn* prog, int nprog, int nscal, Hoisted* h, std::string* err);

// Value of hoisted subexpression j computed on the host, one operation per
// node in T; DSCAL k reads dvals[k] (host values standing for the device
// scalars; NULL when the subexpression has no DSCAL).
double host_scalar_value_f32(const salt_insn* prog, const Hoisted& h, int j, const double* scalars,
                             const double* dvals = nullptr);
double host_scalar_value_f64(const salt_insn* prog, const Hoisted& h, int j, const double* scalars,
                             const double* dvals = nullptr);

// s = +-2^e exactly, with e in the normal range [-1022, 1023]: true and *e.
bool exact_pow2(double s, int* e);
// Pow2Info of an FP64 launch's by-value scalar slots sc[0 .. nscal-1].
Pow2Info pow2_info(const double* sc, int nscal);

// Device code that computes the hoisted slots of canonical program `c`
// (made from h.prog) into canonical scalar slots; user_nscal scalars by
// value, `dscal` device pointers.  False if it would exceed kMaxScalarCode.
bool build_scalar_code(const salt_insn* prog, const Hoisted& h, const Canonical& c, int user_nscal,
                       const double* scalars, const double* const* dscal, ScalarCode* out);

}  // namespace salt
