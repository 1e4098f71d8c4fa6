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
};

// Validates `prog` against nvecs / nscal.  On failure fills `err`.
salt_status analyse(const salt_insn* prog, int nprog, int nvecs, int nscal, Analysis* out,
                    std::string* err);

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

}  // namespace salt
