// Pairwise tensor contraction planner: every contraction of the method is
// written as an einsum-like label string and executed as (at most) one
// permutation per operand, one GEMM and one permutation of the result.
// Operands already laid out as [free, contracted] or [contracted, free] go to
// the GEMM without a copy (transposed operand).
#include <string>
#include "kernels.cuh"

namespace tn {

namespace {

struct Spec { std::string a, b, c; };

bool parse(const char* spec, Spec& s)
{
    std::string t(spec);
    size_t comma = t.find(','), arrow = t.find("->");
    if (comma == std::string::npos || arrow == std::string::npos || arrow < comma) return false;
    s.a = t.substr(0, comma);
    s.b = t.substr(comma + 1, arrow - comma - 1);
    s.c = t.substr(arrow + 2);
    return true;
}

int index_of(const std::string& s, char c) { size_t p = s.find(c); return p == std::string::npos ? -1 : (int)p; }

}  // namespace

int permute_spec(cudaStream_t st, const char* spec, const DT& in, const DT& out)
{
    std::string t(spec);
    size_t arrow = t.find("->");
    if (arrow == std::string::npos) return TN_EINVAL;
    std::string a = t.substr(0, arrow), c = t.substr(arrow + 2);
    if ((int)a.size() != in.rank || c.size() != a.size()) return TN_EINVAL;
    int perm[8];
    for (int j = 0; j < (int)c.size(); ++j) {
        perm[j] = index_of(a, c[j]);
        if (perm[j] < 0) return TN_EINVAL;
    }
    return permute(st, in.p, out.p, in.rank, in.dim, perm);
}

int contract(cudaStream_t st, Arena& ar, const char* spec, const DT& A, const DT& B, const DT& C,
             double alpha, double beta, int kind)
{
    Spec s;
    if (!parse(spec, s)) return TN_EINVAL;
    if ((int)s.a.size() != A.rank || (int)s.b.size() != B.rank || (int)s.c.size() != C.rank) return TN_EINVAL;
    int dim[128];
    for (int i = 0; i < 128; ++i) dim[i] = -1;
    auto setd = [&](const std::string& l, const DT& T) -> bool {
        for (int i = 0; i < (int)l.size(); ++i) {
            int ch = (unsigned char)l[i];
            if (dim[ch] >= 0 && dim[ch] != T.dim[i]) return false;
            dim[ch] = T.dim[i];
        }
        return true;
    };
    if (!setd(s.a, A) || !setd(s.b, B) || !setd(s.c, C)) return TN_EINVAL;
    std::string fa, fb, k;                     // free-A (C order), free-B (C order), contracted (A order)
    for (char ch : s.c) {
        bool ina = index_of(s.a, ch) >= 0, inb = index_of(s.b, ch) >= 0;
        if (ina && inb) return TN_EINVAL;      // batch labels not supported
        if (ina) fa += ch; else if (inb) fb += ch; else return TN_EINVAL;
    }
    for (char ch : s.a) {
        if (index_of(s.c, ch) >= 0) continue;
        if (index_of(s.b, ch) < 0) return TN_EINVAL;   // trace not supported
        k += ch;
    }
    for (char ch : s.b)
        if (index_of(s.c, ch) < 0 && index_of(s.a, ch) < 0) return TN_EINVAL;
    long long M = 1, N = 1, K = 1;
    for (char ch : fa) M *= dim[(unsigned char)ch];
    for (char ch : fb) N *= dim[(unsigned char)ch];
    for (char ch : k) K *= dim[(unsigned char)ch];
    if (M > 0x7fffffff || N > 0x7fffffff || K > 0x7fffffff) return TN_EINVAL;

    size_t mk = ar.mark();
    // operand A as [fa, k] (no transpose) or [k, fa] (transposed)
    const double* pA = A.p;
    bool ta = false;
    if (s.a == fa + k) ta = false;
    else if (s.a == k + fa) ta = true;
    else {
        double* t = ar.take(A.size());
        if (!t) { ar.release(mk); return TN_ENOMEM; }
        DT o = A; o.p = t;
        std::string want = fa + k;
        for (int j = 0; j < (int)want.size(); ++j) o.dim[j] = dim[(unsigned char)want[j]];
        TN_TRY(permute_spec(st, (s.a + "->" + want).c_str(), A, o));
        pA = t;
    }
    // operand B as [k, fb] or [fb, k]
    const double* pB = B.p;
    bool tb = false;
    if (s.b == k + fb) tb = false;
    else if (s.b == fb + k) tb = true;
    else {
        double* t = ar.take(B.size());
        if (!t) { ar.release(mk); return TN_ENOMEM; }
        DT o = B; o.p = t;
        std::string want = k + fb;
        for (int j = 0; j < (int)want.size(); ++j) o.dim[j] = dim[(unsigned char)want[j]];
        TN_TRY(permute_spec(st, (s.b + "->" + want).c_str(), B, o));
        pB = t;
    }
    const int lda = ta ? (int)M : (int)K;
    const int ldb = tb ? (int)K : (int)N;
    if (s.c == fa + fb) {
        TN_TRY(gemm_any(st, ar, kind, ta, tb, (int)M, (int)N, (int)K, alpha, pA, lda, pB, ldb, beta, C.p, (int)N));
    } else {
        if (beta != 0.0) { ar.release(mk); return TN_EINVAL; }
        double* t = ar.take((size_t)M * N);
        if (!t) { ar.release(mk); return TN_ENOMEM; }
        TN_TRY(gemm_any(st, ar, kind, ta, tb, (int)M, (int)N, (int)K, alpha, pA, lda, pB, ldb, 0.0, t, (int)N));
        DT o; o.p = t; o.rank = (int)(fa.size() + fb.size());
        std::string have = fa + fb;
        for (int j = 0; j < o.rank; ++j) o.dim[j] = dim[(unsigned char)have[j]];
        TN_TRY(permute_spec(st, (have + "->" + s.c).c_str(), o, C));
    }
    ar.release(mk);
    return TN_OK;
}

}  // namespace tn
