"""Named postfix programs of the paper's examples and the BLAS-1 set, in the
binding's (name, arg) form (opcodes as in include/salt.h)."""

# Section 2, Figure 1: d = a + (b - c); operands a, b, c, d = 0..3
PROG_D = [("VEC", 0), ("VEC", 1), ("VEC", 2), ("SUB", 0), ("ADD", 0), ("STORE", 3)]
# y = alpha*x + beta*y (Section 5's xAXPY generalised); x, y = 0, 1
PROG_AXPBY = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1)]
# e = alpha*a + beta*b - c o d; a, b, c, d, e = 0..4
PROG_E = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0), ("ADD", 0),
          ("VEC", 2), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4)]
# r <- r - alpha*q ; rho = r.r ; p <- r + beta*p; r, q, p = 0..2
PROG_CG = [("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("SUB", 0), ("STORE", 0), ("VEC", 0), ("SUMSQ", 0),
           ("VEC", 0), ("SCAL", 1), ("VEC", 2), ("SMUL", 0), ("ADD", 0), ("STORE", 2)]
# y = alpha*x (Section 5's out-of-place scaling, sCOPY + sSCAL as one loop)
PROG_SCALE = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 1)]
PROG_DOT = [("VEC", 0), ("VEC", 1), ("DOT", 0)]
PROG_SUMSQ = [("VEC", 0), ("SUMSQ", 0)]
