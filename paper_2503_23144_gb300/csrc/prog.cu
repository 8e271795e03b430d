// Contraction program: primal evaluation and the forward / reverse sweeps.
//
// A slot holds a tensor; an op writes one slot as a sum of terms, each term a
// bilinear contraction (EIN), a permuted copy (PERM), an antisymmetriser (ASYM),
// the particle-particle ladder (LADDER) or the Q map (QMAP); the last two are
// linear in their operand with constant integrals.  The
// transpose rules are the ones of bilinear maps: for C += c A.B,
//   dC += c (dA.B + A.dB),   Abar += c Cbar.B,   Bbar += c A.Cbar
// (holomorphic, no conjugation), a permutation transposes to the inverse
// permutation, the ladder transposes to the ladder built from B^T = conj B, and
// the Q map to its transposed slab contraction.  Primal values and forward
// tangents are kept only where a sweep reads them.
// Tangents and cotangents carry a leading right-hand-side label 'Z'.
#include "prog.h"

#include <algorithm>

namespace {
std::string lhs_a(const std::string& s) { return s.substr(0, s.find(',')); }
std::string lhs_b(const std::string& s) {
    size_t c = s.find(','), a = s.find("->");
    return s.substr(c + 1, a - c - 1);
}
std::string rhs(const std::string& s) { return s.substr(s.find("->") + 2); }
std::string perm_in(const std::string& s) { return s.substr(0, s.find("->")); }

Tensor as5(const Tensor& t, int64_t R, int64_t O, int64_t V) { return t.reshape({R, O, O, V, V}); }
Tensor asq(const Tensor& t, int64_t R, int64_t O, int64_t V) { return t.reshape({R, V, O, O, O}); }
}  // namespace

int Prog::input(std::vector<int64_t> shape) {
    Tensor t;
    t.nd = (int)shape.size();
    for (int k = 0; k < t.nd; ++k) t.d[k] = shape[k];
    val.push_back(t);
    shape0.push_back(shape);
    active.push_back(1);
    is_const.push_back(0);
    inputs.push_back((int)val.size() - 1);
    return (int)val.size() - 1;
}

int Prog::cst(const Tensor& t) {
    val.push_back(t);
    shape0.push_back(t.shape());
    active.push_back(0);
    is_const.push_back(1);
    return (int)val.size() - 1;
}

int Prog::op(std::vector<Term> terms) {
    Op o;
    o.terms = terms;
    bool act = false;
    for (auto& t : terms) {
        if (t.a >= 0 && active[t.a]) act = true;
        if (t.b >= 0 && active[t.b]) act = true;
    }
    val.push_back(Tensor());
    active.push_back(act);
    is_const.push_back(0);
    o.out = (int)val.size() - 1;
    shape0.push_back(out_shape(o));
    ops.push_back(o);
    return o.out;
}

std::vector<int64_t> Prog::out_shape(const Op& op) const {
    const Term& t = op.terms.at(0);
    const std::vector<int64_t>& A = shape0[t.a];
    std::vector<int64_t> sh;
    if (t.kind == TK_LADDER || t.kind == TK_ASYM) return A;
    if (t.kind == TK_QMAP) return {A[2], A[0], A[0], A[0]};  // [O][O][V][V] -> [V][O][O][O]
    if (t.kind == TK_PERM) {
        std::string lx = perm_in(t.spec), ly = rhs(t.spec);
        for (char c : ly) sh.push_back(A[lx.find(c)]);
        return sh;
    }
    std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
    const std::vector<int64_t>& B = shape0[t.b];
    for (char c : lc) {
        size_t p = la.find(c);
        if (p != std::string::npos) sh.push_back(A[p]);
        else sh.push_back(B[lb.find(c)]);
    }
    return sh;
}

// view of an unbatched tensor repeated RB times along a new leading dim (stride 0)
static Tensor broadcast(const Tensor& t, int64_t R) {
    Tensor v = t;
    for (int k = v.nd; k > 0; --k) {
        v.d[k] = v.d[k - 1];
        v.s[k] = v.s[k - 1];
    }
    v.d[0] = R;
    v.s[0] = 0;
    v.nd = t.nd + 1;
    return v;
}

void Prog::apply_term(Dev& D, const Term& t, cplx beta, Tensor& out, int prec) {
    const cplx c = t.c;
    if (t.kind == TK_EIN) {
        std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
        std::string za = zp(t.a), zb = zp(t.b);
        bool out_batched = RB > 0 && (active[t.a] || active[t.b] || out.nd > (int)lc.size());
        if (RB > 0 && za.empty() && zb.empty() && out_batched) {
            // both operands constant, batched output: compute once and broadcast
            Tensor tmp = ein_new(D, t.spec, c, val[t.a], false, val[t.b], false, prec);
            axpby(D, mkc(1.0), broadcast(tmp, RB), false, beta, out);
            return;
        }
        std::string zc = out_batched ? "Z" : "";
        ein(D, za + la + "," + zb + lb + "->" + zc + lc, c, val[t.a], false, val[t.b], false, beta, out, prec);
    } else if (t.kind == TK_PERM) {
        std::string lx = perm_in(t.spec), ly = rhs(t.spec);
        bool out_batched = RB > 0 && out.nd > (int)ly.size();
        if (out_batched && zp(t.a).empty()) {
            Tensor x = broadcast(val[t.a], RB);
            perm_axpby(D, "Z" + lx + "->Z" + ly, c, x, beta, out);
        } else {
            std::string z = out_batched ? "Z" : "";
            perm_axpby(D, z + lx + "->" + z + ly, c, val[t.a], beta, out);
        }
    } else if (t.kind == TK_ASYM) {
        REQUIRE(RB == 0 || active[t.a], "asym term on a constant in a batched evaluation");
        asym_axpby(D, asym_mode(t), c, val[t.a], beta, out);
    } else if (t.kind == TK_QMAP) {
        int64_t R = (RB > 0 && active[t.a]) ? RB : 1;
        Tensor x = as5(val[t.a], R, O, V);
        Tensor q = asq(out, R, O, V);
        qmap(D, *lad, x, c, beta, q, prec);
    } else {
        int64_t R = (RB > 0 && active[t.a]) ? RB : 1;
        Tensor x = as5(val[t.a], R, O, V);
        Tensor z = as5(out, R, O, V);
        ladder(D, *lad, x, c, beta, z, false, prec);
    }
}

void Prog::eval(Dev& D, const std::vector<Tensor>& in, int prec, bool batched) {
    if (in.size() != inputs.size()) throw LrccError(LRCC_EINVAL, "program input count");
    RB = batched ? in.at(0).d[0] : 0;
    for (size_t k = 0; k < in.size(); ++k) {
        std::vector<int64_t> want = shape0[inputs[k]];
        if (batched) want.insert(want.begin(), RB);
        REQUIRE(in[k].shape() == want, "program input shape");
        val[inputs[k]] = in[k];
    }
    // a slot's value is dropped after its last use here unless the sweeps read
    // it (needs_value), it is an output, an input or a constant
    build_need();
    const int n = (int)val.size();
    std::vector<int> last(n, -1);
    for (int k = 0; k < (int)ops.size(); ++k)
        for (auto& t : ops[k].terms) {
            if (t.a >= 0) last[t.a] = k;
            if (t.b >= 0) last[t.b] = k;
        }
    std::vector<char> keep(n, 0);
    for (int s = 0; s < n; ++s) keep[s] = is_const[s] || need_val_[s];
    for (int s : inputs) keep[s] = 1;
    for (int s : outputs) keep[s] = 1;
    for (int k = 0; k < (int)ops.size(); ++k) {
        const Op& o = ops[k];
        std::vector<int64_t> sh = shape0[o.out];
        if (RB > 0 && active[o.out]) sh.insert(sh.begin(), RB);
        Tensor out = empty(D, sh);
        bool first = true;
        for (auto& t : o.terms) {
            apply_term(D, t, first ? mkc(0.0) : mkc(1.0), out, prec);
            first = false;
        }
        val[o.out] = out;
        for (auto& t : o.terms)
            for (int s : {t.a, t.b})
                if (s >= 0 && last[s] == k && !keep[s]) val[s] = Tensor();
        if (last[o.out] < 0 && !keep[o.out]) val[o.out] = Tensor();
    }
}

void Prog::build_need() {
    if (need_val_.size() == val.size()) return;
    need_val_.assign(val.size(), 0);
    for (auto& o : ops)
        for (auto& t : o.terms) {
            if (t.kind != TK_EIN) continue;
            if (active[t.b]) need_val_[t.a] = 1;  // tangents/adjoints of t.b read the value of t.a
            if (active[t.a]) need_val_[t.b] = 1;
        }
}

bool Prog::needs_value(int slot) const {
    return slot >= 0 && slot < (int)need_val_.size() && need_val_[slot];
}

std::vector<Tensor> Prog::jvp(Dev& D, const std::vector<Tensor>& tin, const std::vector<int>& outs, int prec) {
    const int n = (int)val.size();
    std::vector<Tensor> tan(n);
    int64_t R = tin.at(0).d[0];
    REQUIRE(RB == 0 || RB == R, "jvp: tangent batch must match the primal batch");
    for (size_t k = 0; k < inputs.size(); ++k) tan[inputs[k]] = tin[k];
    std::vector<int> last(n, -1);
    for (int k = 0; k < (int)ops.size(); ++k)
        for (auto& t : ops[k].terms) {
            if (t.a >= 0) last[t.a] = k;
            if (t.b >= 0) last[t.b] = k;
        }
    for (int o : outs) last[o] = (int)ops.size();
    for (size_t k = 0; k < inputs.size(); ++k) last[inputs[k]] = (int)ops.size();
    // only ops whose result reaches a requested output
    std::vector<char> need(n, 0);
    for (int o : outs) need[o] = 1;
    for (int k = (int)ops.size() - 1; k >= 0; --k) {
        if (!need[ops[k].out]) continue;
        for (auto& t : ops[k].terms) {
            if (t.a >= 0) need[t.a] = 1;
            if (t.b >= 0) need[t.b] = 1;
        }
    }
    for (int k = 0; k < (int)ops.size(); ++k) {
        const Op& o = ops[k];
        if (!active[o.out] || !need[o.out]) continue;
        std::vector<int64_t> sh = shape0[o.out];
        sh.insert(sh.begin(), R);
        Tensor out = empty(D, sh);
        bool first = true;
        auto beta = [&]() { cplx b = first ? mkc(0.0) : mkc(1.0); first = false; return b; };
        for (auto& t : o.terms) {
            if (t.kind == TK_EIN) {
                std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
                if (active[t.a])
                    ein(D, "Z" + la + "," + zp(t.b) + lb + "->Z" + lc, t.c, tan[t.a], false, val[t.b], false, beta(), out, prec);
                if (active[t.b])
                    ein(D, zp(t.a) + la + ",Z" + lb + "->Z" + lc, t.c, val[t.a], false, tan[t.b], false, beta(), out, prec);
            } else if (t.kind == TK_PERM) {
                if (active[t.a]) perm_axpby(D, "Z" + perm_in(t.spec) + "->Z" + rhs(t.spec), t.c, tan[t.a], beta(), out);
            } else if (t.kind == TK_ASYM) {
                if (active[t.a]) asym_axpby(D, asym_mode(t), t.c, tan[t.a], beta(), out);
            } else if (t.kind == TK_QMAP) {
                if (active[t.a]) {
                    Tensor x = as5(tan[t.a], R, O, V), q = asq(out, R, O, V);
                    qmap(D, *lad, x, t.c, beta(), q, prec);
                }
            } else {
                if (active[t.a]) {
                    Tensor x = as5(tan[t.a], R, O, V), z = as5(out, R, O, V);
                    ladder(D, *lad, x, t.c, beta(), z, false, prec);
                }
            }
        }
        if (first) fill(D, out, mkc(0.0));
        tan[o.out] = out;
        for (auto& t : o.terms) {
            if (t.a >= 0 && last[t.a] == k) tan[t.a] = Tensor();
            if (t.b >= 0 && last[t.b] == k) tan[t.b] = Tensor();
        }
    }
    std::vector<Tensor> res;
    for (int o : outs) res.push_back(tan[o]);
    return res;
}

std::vector<Tensor> Prog::vjp(Dev& D, const std::vector<Tensor>& cot, const std::vector<int>& outs, int prec) {
    const int n = (int)val.size();
    std::vector<Tensor> adj(n);
    std::vector<char> has(n, 0);
    int64_t R = -1;
    for (size_t k = 0; k < outs.size(); ++k) {
        if (cot[k].p == nullptr) continue;
        adj[outs[k]] = cot[k];
        has[outs[k]] = 1;
        R = cot[k].d[0];
    }
    if (R < 0) throw LrccError(LRCC_EINVAL, "vjp: all cotangents are zero");
    REQUIRE(RB == 0 || RB == R, "vjp: cotangent batch must match the primal batch");
    auto acc = [&](int slot, auto&& write) {
        if (!active[slot]) return;
        if (!has[slot]) {
            std::vector<int64_t> sh = shape0[slot];
            sh.insert(sh.begin(), R);
            adj[slot] = empty(D, sh);
            write(adj[slot], mkc(0.0));
            has[slot] = 1;
        } else {
            write(adj[slot], mkc(1.0));
        }
    };
    for (int k = (int)ops.size() - 1; k >= 0; --k) {
        const Op& o = ops[k];
        if (!active[o.out] || !has[o.out]) continue;
        Tensor cb = adj[o.out];
        for (auto& t : o.terms) {
            if (t.kind == TK_EIN) {
                std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
                if (active[t.a])
                    acc(t.a, [&](Tensor& dst, cplx b) {
                        ein(D, "Z" + lc + "," + zp(t.b) + lb + "->Z" + la, t.c, cb, false, val[t.b], false, b, dst, prec);
                    });
                if (active[t.b])
                    acc(t.b, [&](Tensor& dst, cplx b) {
                        ein(D, zp(t.a) + la + ",Z" + lc + "->Z" + lb, t.c, val[t.a], false, cb, false, b, dst, prec);
                    });
            } else if (t.kind == TK_PERM) {
                if (active[t.a])
                    acc(t.a, [&](Tensor& dst, cplx b) {
                        perm_axpby(D, "Z" + rhs(t.spec) + "->Z" + perm_in(t.spec), t.c, cb, b, dst);
                    });
            } else if (t.kind == TK_ASYM) {
                if (active[t.a])
                    acc(t.a, [&](Tensor& dst, cplx b) { asym_axpby(D, asym_mode(t), t.c, cb, b, dst); });
            } else if (t.kind == TK_QMAP) {
                if (active[t.a])
                    acc(t.a, [&](Tensor& dst, cplx b) {
                        Tensor q = asq(cb, R, O, V), z = as5(dst, R, O, V);
                        qmap_t(D, *lad, q, t.c, b, z, prec);
                    });
            } else {
                if (active[t.a])
                    acc(t.a, [&](Tensor& dst, cplx b) {
                        Tensor x = as5(cb, R, O, V), z = as5(dst, R, O, V);
                        ladder(D, *lad, x, t.c, b, z, true, prec);
                    });
            }
        }
        bool is_in = std::find(inputs.begin(), inputs.end(), o.out) != inputs.end();
        if (!is_in) adj[o.out] = Tensor();
    }
    std::vector<Tensor> res;
    for (int s : inputs) {
        if (!has[s]) {
            std::vector<int64_t> sh = shape0[s];
            sh.insert(sh.begin(), R);
            res.push_back(zeros(D, sh));
        } else {
            res.push_back(adj[s]);
        }
    }
    return res;
}

std::vector<Tensor> Prog::jvp_of_vjp(Dev& D, const std::vector<Tensor>& tin, const std::vector<Tensor>& cot,
                                     const std::vector<int>& outs, int prec) {
    REQUIRE(RB == 0, "jvp_of_vjp needs the unbatched primal");
    const int n = (int)val.size();
    const int64_t R = tin.at(0).d[0];
    // 1. tangents of every active slot; kept only where the reverse sweep
    // reads them (operands of contractions with another active operand)
    build_need();
    std::vector<Tensor> tan(n);
    for (size_t k = 0; k < inputs.size(); ++k) tan[inputs[k]] = tin[k];
    std::vector<int> lastf(n, -1);
    for (int k = 0; k < (int)ops.size(); ++k)
        for (auto& t : ops[k].terms) {
            if (t.a >= 0) lastf[t.a] = k;
            if (t.b >= 0) lastf[t.b] = k;
        }
    auto drop_tangents = [&](const Op& o, int k) {
        for (auto& t : o.terms)
            for (int s : {t.a, t.b})
                if (s >= 0 && lastf[s] == k && !need_val_[s] &&
                    std::find(inputs.begin(), inputs.end(), s) == inputs.end())
                    tan[s] = Tensor();
    };
    for (int k = 0; k < (int)ops.size(); ++k) {
        const Op& o = ops[k];
        if (!active[o.out]) continue;
        std::vector<int64_t> sh = shape0[o.out];
        sh.insert(sh.begin(), R);
        Tensor out = empty(D, sh);
        bool first = true;
        auto beta = [&]() { cplx b = first ? mkc(0.0) : mkc(1.0); first = false; return b; };
        for (auto& t : o.terms) {
            if (t.kind == TK_EIN) {
                std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
                if (active[t.a]) ein(D, "Z" + la + "," + lb + "->Z" + lc, t.c, tan[t.a], false, val[t.b], false, beta(), out, prec);
                if (active[t.b]) ein(D, la + ",Z" + lb + "->Z" + lc, t.c, val[t.a], false, tan[t.b], false, beta(), out, prec);
            } else if (t.kind == TK_PERM) {
                if (active[t.a]) perm_axpby(D, "Z" + perm_in(t.spec) + "->Z" + rhs(t.spec), t.c, tan[t.a], beta(), out);
            } else if (t.kind == TK_ASYM) {
                if (active[t.a]) asym_axpby(D, asym_mode(t), t.c, tan[t.a], beta(), out);
            } else if (t.kind == TK_QMAP) {
                if (active[t.a]) {
                    Tensor x = as5(tan[t.a], R, O, V), q = asq(out, R, O, V);
                    qmap(D, *lad, x, t.c, beta(), q, prec);
                }
            } else if (active[t.a]) {
                Tensor x = as5(tan[t.a], R, O, V), z = as5(out, R, O, V);
                ladder(D, *lad, x, t.c, beta(), z, false, prec);
            }
        }
        if (first) fill(D, out, mkc(0.0));
        tan[o.out] = out;
        drop_tangents(o, k);
        if (lastf[o.out] < 0 && !need_val_[o.out]) tan[o.out] = Tensor();
    }
    // 2. adjoints (unbatched: leading dim 1 dropped) and 3. their tangents, in one reverse sweep
    std::vector<Tensor> adj(n), dadj(n);
    for (size_t k = 0; k < outs.size(); ++k)
        if (cot[k].p) adj[outs[k]] = cot[k].index(0);
    auto acc1 = [&](int slot, auto&& write) {  // unbatched adjoint accumulation
        if (!active[slot]) return;
        if (!adj[slot].p) {
            adj[slot] = empty(D, shape0[slot]);
            write(adj[slot], mkc(0.0));
        } else {
            write(adj[slot], mkc(1.0));
        }
    };
    auto accR = [&](int slot, auto&& write) {  // batched tangent-of-adjoint accumulation
        if (!active[slot]) return;
        if (!dadj[slot].p) {
            std::vector<int64_t> sh = shape0[slot];
            sh.insert(sh.begin(), R);
            dadj[slot] = empty(D, sh);
            write(dadj[slot], mkc(0.0));
        } else {
            write(dadj[slot], mkc(1.0));
        }
    };
    for (int k = (int)ops.size() - 1; k >= 0; --k) {
        const Op& o = ops[k];
        if (!active[o.out]) continue;
        Tensor cb = adj[o.out], dcb = dadj[o.out];
        if (!cb.p && !dcb.p) continue;
        for (auto& t : o.terms) {
            if (t.kind == TK_EIN) {
                std::string la = lhs_a(t.spec), lb = lhs_b(t.spec), lc = rhs(t.spec);
                if (active[t.a]) {
                    if (cb.p)
                        acc1(t.a, [&](Tensor& dst, cplx b) {
                            ein(D, lc + "," + lb + "->" + la, t.c, cb, false, val[t.b], false, b, dst, prec);
                        });
                    if (dcb.p)
                        accR(t.a, [&](Tensor& dst, cplx b) {
                            ein(D, "Z" + lc + "," + lb + "->Z" + la, t.c, dcb, false, val[t.b], false, b, dst, prec);
                        });
                    if (cb.p && active[t.b])
                        accR(t.a, [&](Tensor& dst, cplx b) {
                            ein(D, lc + ",Z" + lb + "->Z" + la, t.c, cb, false, tan[t.b], false, b, dst, prec);
                        });
                }
                if (active[t.b]) {
                    if (cb.p)
                        acc1(t.b, [&](Tensor& dst, cplx b) {
                            ein(D, la + "," + lc + "->" + lb, t.c, val[t.a], false, cb, false, b, dst, prec);
                        });
                    if (dcb.p)
                        accR(t.b, [&](Tensor& dst, cplx b) {
                            ein(D, la + ",Z" + lc + "->Z" + lb, t.c, val[t.a], false, dcb, false, b, dst, prec);
                        });
                    if (cb.p && active[t.a])
                        accR(t.b, [&](Tensor& dst, cplx b) {
                            ein(D, "Z" + la + "," + lc + "->Z" + lb, t.c, tan[t.a], false, cb, false, b, dst, prec);
                        });
                }
            } else if (t.kind == TK_ASYM) {
                if (!active[t.a]) continue;
                if (cb.p) acc1(t.a, [&](Tensor& dst, cplx b) { asym_axpby(D, asym_mode(t), t.c, cb, b, dst); });
                if (dcb.p) accR(t.a, [&](Tensor& dst, cplx b) { asym_axpby(D, asym_mode(t), t.c, dcb, b, dst); });
            } else if (t.kind == TK_PERM) {
                if (!active[t.a]) continue;
                std::string lx = perm_in(t.spec), ly = rhs(t.spec);
                if (cb.p)
                    acc1(t.a, [&](Tensor& dst, cplx b) { perm_axpby(D, ly + "->" + lx, t.c, cb, b, dst); });
                if (dcb.p)
                    accR(t.a, [&](Tensor& dst, cplx b) { perm_axpby(D, "Z" + ly + "->Z" + lx, t.c, dcb, b, dst); });
            } else if (t.kind == TK_QMAP) {
                if (!active[t.a]) continue;
                if (cb.p)
                    acc1(t.a, [&](Tensor& dst, cplx b) {
                        Tensor q = asq(cb, 1, O, V), z = as5(dst, 1, O, V);
                        qmap_t(D, *lad, q, t.c, b, z, prec);
                    });
                if (dcb.p)
                    accR(t.a, [&](Tensor& dst, cplx b) {
                        Tensor q = asq(dcb, R, O, V), z = as5(dst, R, O, V);
                        qmap_t(D, *lad, q, t.c, b, z, prec);
                    });
            } else {
                if (!active[t.a]) continue;
                if (cb.p)
                    acc1(t.a, [&](Tensor& dst, cplx b) {
                        Tensor x = as5(cb, 1, O, V), z = as5(dst, 1, O, V);
                        ladder(D, *lad, x, t.c, b, z, true, prec);
                    });
                if (dcb.p)
                    accR(t.a, [&](Tensor& dst, cplx b) {
                        Tensor x = as5(dcb, R, O, V), z = as5(dst, R, O, V);
                        ladder(D, *lad, x, t.c, b, z, true, prec);
                    });
            }
        }
        bool is_in = std::find(inputs.begin(), inputs.end(), o.out) != inputs.end();
        if (!is_in) {
            adj[o.out] = Tensor();
            dadj[o.out] = Tensor();
            tan[o.out] = Tensor();
        }
    }
    std::vector<Tensor> res;
    for (int s : inputs) {
        if (!dadj[s].p) {
            std::vector<int64_t> sh = shape0[s];
            sh.insert(sh.begin(), R);
            res.push_back(zeros(D, sh));
        } else {
            res.push_back(dadj[s]);
        }
    }
    return res;
}

// ---------------------------------------------------------------------------
// integrals and the CCSD residual
// ---------------------------------------------------------------------------
Tensor anti_block(Dev& D, const Tensor& B, int64_t p0, int64_t np, int64_t q0, int64_t nq, int64_t r0, int64_t nr,
                  int64_t s0, int64_t ns) {
    auto sub = [&](int64_t x0, int64_t nx, int64_t y0, int64_t ny) { return B.slice(1, x0, nx).slice(2, y0, ny); };
    Tensor out = empty(D, {np, nq, nr, ns});
    // <pq|rs> = sum_L B^L_pr B^L_qs ;  <pq|sr> = sum_L B^L_ps B^L_qr
    ein(D, "Lpr,Lqs->pqrs", mkc(1.0), sub(p0, np, r0, nr), false, sub(q0, nq, s0, ns), false, mkc(0.0), out);
    ein(D, "Lps,Lqr->pqrs", mkc(-1.0), sub(p0, np, s0, ns), false, sub(q0, nq, r0, nr), false, mkc(1.0), out);
    return out;
}

// Spin-orbital CCSD (Stanton, Gauss, Watts, Bartlett 1991 intermediates) for a
// general Fock matrix, with the driver terms in their general complex form
// (<ab||ij>, f_ai).  Terms are regrouped for a density-fitted ladder:
//   1/2 sum_ef tau_ij^ef W_abef = ladder(tau) - 1/2 P(ab) sum_m t_m^b Q_amij
//                                 + 1/8 sum_mn tau_mn^ab P_mnij,
// Q_amij = sum_ef <am||ef> tau_ij^ef, P_mnij = sum_ef <mn||ef> tau_ij^ef, and the
// last piece is merged into W_mnij (its 1/4 P_mnij becomes 1/2 P_mnij).
// Integrals with three virtual indices are contracted through the factor,
// <pq|rs> = sum_L B^L_pr B^L_qs, so that no O V^3 block is formed:
//   sum_mf t_m^f <ma||fe> = sum_L g_L B^L_ae - sum_Lm B^L_me G^L_am,
//   sum_mef t_im^ef <ma||ef> = sum_Lf U^L_if B^L_af - sum_Le U'^L_ie B^L_ae,
//   sum_f t_j^f <mb||ef> = sum_L (B^L_me G^L_bj - H^L_mj B^L_be),
//   sum_e t_i^e <ab||ej> = sum_L (G^L_ai B^L_bj - B^L_aj G^L_bi),
// with G^L_ai = sum_e B^L_ae t_i^e, g_L = sum_mf B^L_mf t_m^f, H^L_mj =
// sum_f B^L_mf t_j^f, U^L_if = sum_me t_im^ef B^L_me, U'^L_ie = sum_mf t_im^ef
// B^L_mf, and Q from <am||ef> assembled in slabs (the Q map).  The doubles
// residual is accumulated in a chain of ops so that each group of terms is
// released as soon as it is added.
void build_ccsd(CCProg& cp, const Ham& H, LadderCtx* lad) {
    Prog& P = cp.P;
    P.lad = lad;
    int64_t O = H.foo.d[0], V = H.fvv.d[0];
    P.O = (int)O;
    P.V = (int)V;
    const bool w = H.w;
    int t1 = P.input({O, V}), t2 = P.input({O, O, V, V});
    cp.t1 = t1;
    cp.t2 = t2;
    int foo = P.cst(H.foo), fov = P.cst(H.fov), fvo = P.cst(H.fvo), fvv = P.cst(H.fvv);
    int oooo = -1, ooov = -1, oovo = -1, ovoo = -1, oovv = -1, vvoo = -1, ovov = -1, ovvo = -1;
    int Bov = -1, Bvo = -1, Bvv = -1;
    if (w) {
        oooo = P.cst(H.oooo); ooov = P.cst(H.ooov); oovo = P.cst(H.oovo); ovoo = P.cst(H.ovoo);
        oovv = P.cst(H.oovv); vvoo = P.cst(H.vvoo); ovov = P.cst(H.ovov); ovvo = P.cst(H.ovvo);
        Bov = P.cst(H.Bov); Bvo = P.cst(H.Bvo); Bvv = P.cst(H.Bvv);
    }
    int taut = P.op({PERM(1, "ijab->ijab", t2), EIN(0.5, "ia,jb->ijab", t1, t1), EIN(-0.5, "ib,ja->ijab", t1, t1)});
    int tau = P.op({PERM(1, "ijab->ijab", t2), EIN(1, "ia,jb->ijab", t1, t1), EIN(-1, "ib,ja->ijab", t1, t1)});
    int G = -1, Hm = -1;
    if (w) {
        G = P.op({EIN(1, "ie,Lae->Lai", t1, Bvv)});
        Hm = P.op({EIN(1, "jf,Lmf->Lmj", t1, Bov)});
    }

    std::vector<Term> fae = {PERM(1, "ae->ae", fvv), EIN(-0.5, "me,ma->ae", fov, t1)};
    std::vector<Term> fmi = {PERM(1, "mi->mi", foo), EIN(0.5, "ie,me->mi", t1, fov)};
    std::vector<Term> fme = {PERM(1, "me->me", fov)};
    if (w) {
        int g1 = P.op({EIN(1, "mf,Lmf->L", t1, Bov)});
        fae.push_back(EIN(1, "L,Lae->ae", g1, Bvv));
        fae.push_back(EIN(-1, "Lme,Lam->ae", Bov, G));
        fae.push_back(EIN(-0.5, "mnaf,mnef->ae", taut, oovv));
        fmi.push_back(EIN(1, "ne,mnie->mi", t1, ooov));
        fmi.push_back(EIN(0.5, "inef,mnef->mi", taut, oovv));
        fme.push_back(EIN(1, "nf,mnef->me", t1, oovv));
    }
    int Fae = P.op(fae), Fmi = P.op(fmi), Fme = P.op(fme);

    std::vector<Term> r1 = {PERM(1, "ai->ia", fvo), EIN(1, "ie,ae->ia", t1, Fae), EIN(-1, "ma,mi->ia", t1, Fmi),
                            EIN(1, "imae,me->ia", t2, Fme)};
    if (w) {
        int U = P.op({EIN(1, "imef,Lme->Lif", t2, Bov)});
        int U2 = P.op({EIN(1, "imef,Lmf->Lie", t2, Bov)});
        r1.push_back(EIN(-1, "nf,naif->ia", t1, ovov));
        r1.push_back(EIN(-0.5, "Lif,Laf->ia", U, Bvv));
        r1.push_back(EIN(0.5, "Lie,Lae->ia", U2, Bvv));
        r1.push_back(EIN(-0.5, "mnae,nmei->ia", t2, oovo));
    }
    cp.R1 = P.op(r1);

    int Fbe = P.op({PERM(1, "be->be", Fae), EIN(-0.5, "mb,me->be", t1, Fme)});
    int Fmj = P.op({PERM(1, "mj->mj", Fmi), EIN(0.5, "je,me->mj", t1, Fme)});
    int Xa = P.op({EIN(1, "ijae,be->ijab", t2, Fbe)});
    int Xb = P.op({EIN(1, "imab,mj->ijab", t2, Fmj)});
    std::vector<Term> r2a = {ASYM(1, Xa, 2), ASYM(-1, Xb, 1)};
    if (!w) {
        cp.R2 = P.op(r2a);
    } else {
        r2a.push_back(PERM(1, "abij->ijab", vvoo));
        int R2a = P.op(r2a);
        int Xw = P.op({EIN(1, "je,mnie->mnij", t1, ooov)});
        int Pm = P.op({EIN(1, "ijef,mnef->mnij", tau, oovv)});
        int Wmn = P.op({PERM(1, "mnij->mnij", oooo), PERM(1, "mnij->mnij", Xw), PERM(-1, "mnij->mnji", Xw),
                        PERM(0.5, "mnij->mnij", Pm)});
        int Q = P.op({QMAP(1, tau)});
        int S = P.op({EIN(1, "amij,mb->ijab", Q, t1)});
        int R2b = P.op({PERM(1, "ijab->ijab", R2a), EIN(0.5, "mnab,mnij->ijab", tau, Wmn), LADDER(1, tau),
                        ASYM(-0.5, S, 2)});
        int Zt = P.op({PERM(0.5, "jnfb->jnfb", t2), EIN(1, "jf,nb->jnfb", t1, t1)});
        int Wmbej = P.op({PERM(1, "mbej->mbej", ovvo), EIN(1, "Lme,Lbj->mbej", Bov, G),
                          EIN(-1, "Lmj,Lbe->mbej", Hm, Bvv), EIN(-1, "nb,mnej->mbej", t1, oovo),
                          EIN(-1, "jnfb,mnef->mbej", Zt, oovv)});
        int tmp = P.op({EIN(1, "ie,mbej->mbij", t1, ovvo)});
        int ring = P.op({EIN(1, "imae,mbej->ijab", t2, Wmbej), EIN(-1, "ma,mbij->ijab", t1, tmp)});
        int R2c = P.op({PERM(1, "ijab->ijab", R2b), ASYM(1, ring, 3)});
        int t3 = P.op({EIN(1, "Lai,Lbj->ijab", G, Bvo), EIN(-1, "Laj,Lbi->ijab", Bvo, G)});
        int t4 = P.op({EIN(1, "ma,mbij->ijab", t1, ovoo)});
        cp.R2 = P.op({PERM(1, "ijab->ijab", R2c), ASYM(1, t3, 1), ASYM(-1, t4, 2)});
    }

    std::vector<Term> e = {EIN(1, "ia,ia->", fov, t1)};
    if (w) {
        e.push_back(EIN(0.25, "ijab,ijab->", oovv, t2));
        int Ej = P.op({EIN(1, "ijab,ia->jb", oovv, t1)});
        e.push_back(EIN(0.5, "jb,jb->", Ej, t1));
    }
    cp.E = P.op(e);
    P.outputs = {cp.R1, cp.R2, cp.E};
}
