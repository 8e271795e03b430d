// Contraction program ("tape") for the coupled-cluster residual, with the
// forward (Jacobian-vector) and reverse (transpose-Jacobian) sweeps that give
// sigma = A X and A^T lambda over R right-hand sides at once.
#pragma once
#include "lrcc_internal.h"

enum TermKind { TK_EIN = 0, TK_PERM = 1, TK_LADDER = 2, TK_ASYM = 3, TK_QMAP = 4 };

struct Term {
    TermKind kind;
    cplx c;
    std::string spec;  // "ab,bc->ac" (EIN) or "ab->ba" (PERM)
    int a = -1, b = -1;
};

inline Term EIN(double c, const char* spec, int a, int b) { return Term{TK_EIN, mkc(c), spec, a, b}; }
inline Term PERM(double c, const char* spec, int a) { return Term{TK_PERM, mkc(c), spec, a, -1}; }
inline Term LADDER(double c, int a) { return Term{TK_LADDER, mkc(c), "", a, -1}; }
// Q_amij = sum_ef <am||ef> X_ij^ef of an [O][O][V][V] slot (output [V][O][O][O]),
// linear in X with constant integrals assembled from B in slabs over a
inline Term QMAP(double c, int a) { return Term{TK_QMAP, mkc(c), "", a, -1}; }
// antisymmetriser of an [O][O][V][V] slot: mode 1 P(ij), 2 P(ab), 3 P(ij)P(ab)
// (the operand index b carries the mode; it is not a slot)
inline Term ASYM(double c, int a, int mode) { return Term{TK_ASYM, mkc(c), "", a, -1 - mode}; }
inline int asym_mode(const Term& t) { return -1 - t.b; }

struct Op {
    int out;
    std::vector<Term> terms;
};

struct Prog {
    std::vector<Tensor> val;        // primal value of each slot
    std::vector<std::vector<int64_t>> shape0;  // unbatched shape of each slot
    std::vector<char> active;       // slot depends on the inputs
    std::vector<char> is_const;     // slot is a fixed constant tensor
    std::vector<Op> ops;
    std::vector<int> inputs;        // input slots (amplitudes)
    std::vector<int> outputs;       // slots read after evaluation (residuals, energy)
    LadderCtx* lad = nullptr;
    int O = 0, V = 0;
    int64_t RB = 0;                 // primal batch: 0 = unbatched, else leading dim of active slots

    int input(std::vector<int64_t> shape);
    int cst(const Tensor& t);
    int op(std::vector<Term> terms);

    // primal evaluation for the given input values; with batched = true every
    // input carries a leading batch dimension and so does every active slot
    void eval(Dev& D, const std::vector<Tensor>& in, int prec, bool batched = false);
    // forward sweep: tangents of inputs [R][...] -> tangents of `outs`
    std::vector<Tensor> jvp(Dev& D, const std::vector<Tensor>& tin, const std::vector<int>& outs, int prec);
    // reverse sweep: cotangents of `outs` [R][...] (undefined tensor = zero)
    // -> cotangents of the inputs (holomorphic transpose, no conjugation)
    std::vector<Tensor> vjp(Dev& D, const std::vector<Tensor>& cot, const std::vector<int>& outs, int prec);
    // forward-over-reverse: the directional derivative, along the input
    // tangents tin [R][...], of the reverse sweep with fixed cotangents cot
    // (leading dim 1, shared by all R directions).  Returns [R][...] per input.
    // Needs the unbatched primal (eval with batched = false).
    std::vector<Tensor> jvp_of_vjp(Dev& D, const std::vector<Tensor>& tin, const std::vector<Tensor>& cot,
                                   const std::vector<int>& outs, int prec);

    // slot whose primal value a sweep reads: an operand of a contraction
    // whose other operand depends on the inputs (the only terms whose
    // derivative is not a fixed linear map)
    bool needs_value(int slot) const;

  private:
    std::vector<int64_t> out_shape(const Op& op) const;
    std::vector<char> need_val_;    // cache of needs_value, built on first use
    void build_need();
    // label prefix of a slot's primal value ("Z" when batched)
    std::string zp(int slot) const { return (RB > 0 && active[slot]) ? "Z" : ""; }
    void apply_term(Dev& D, const Term& t, cplx beta, Tensor& out, int prec);
};

// Hamiltonian blocks on the device.  <pq||rs> = <pq|rs> - <pq|sr>.  The
// blocks with three virtual indices (O V^3 elements) are never formed: terms
// that need them contract through the factor blocks Bov [L][O][V] (B^L_me),
// Bvo [L][V][O] and Bvv [L][V][V].
struct Ham {
    bool w = false;  // two-body part present
    Tensor foo, fov, fvo, fvv;
    Tensor oooo, ooov, oovo, ovoo, oovv, vvoo, ovov, ovvo;
    Tensor Bov, Bvo, Bvv;
};

// slots of a CCSD residual program
struct CCProg {
    Prog P;
    int t1 = -1, t2 = -1;   // inputs
    int R1 = -1, R2 = -1, E = -1;
};

// Build the spin-orbital CCSD residual R(T), energy E(T) (general Fock
// matrix; two-body terms only if H.w).
void build_ccsd(CCProg& cp, const Ham& H, LadderCtx* lad);

// Antisymmetrised block <PQ||RS> from B [L][N][N]; ranges (start, length).
Tensor anti_block(Dev& D, const Tensor& B, int64_t p0, int64_t np, int64_t q0, int64_t nq, int64_t r0, int64_t nr,
                  int64_t s0, int64_t ns);
