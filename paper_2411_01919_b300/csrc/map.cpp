// map.cpp -- the polygon map manager of Sec. III-E (host code, no GPU):
// polygons observed in each frame are moved into the map frame with the
// frame's pose, matched against the map (overlapping footprints, centroid
// heights within the drift tolerance, Eq. 4-5), the matches give one
// measurement of the vertical drift for a scalar Kalman filter (Eq. 6-10),
// the new polygons are shifted by the updated drift estimate and then merged
// into the polygons they matched or added to the map.
//
// Only horizontal polygons (treads, floor, landings: the ones the drift is
// measured on and a gait planner steps on) enter the map.  Footprints are
// convex hulls in the map's x-y plane.  The map is the height reference the
// drift is measured against: a merge extends the map polygon's footprint to
// the hull of both and keeps its height (averaging the heights would let the
// drift leak into the map, which then absorbs part of every later offset).
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pm.h"

namespace pm {
pm_status set_last_error(pm_status s, const char *msg);   // pm_api.cu
}

namespace {

struct Poly {
    std::vector<double> x, y;   // convex footprint, counter-clockwise, no repeated vertex
    double z = 0.0;             // height of the centroid (drift-compensated)
    double area = 0.0;
    int observations = 0;
};

double shoelace(const std::vector<double> &x, const std::vector<double> &y)
{
    double a = 0.0;
    const size_t n = x.size();
    for (size_t i = 0; i < n; ++i) {
        const size_t j = (i + 1) % n;
        a += x[i] * y[j] - x[j] * y[i];
    }
    return 0.5 * a;
}

double cross(double ox, double oy, double ax, double ay, double bx, double by)
{
    return (ax - ox) * (by - oy) - (ay - oy) * (bx - ox);
}

// Convex hull (Andrew's monotone chain), counter-clockwise, collinear points dropped.
void convex_hull(std::vector<std::pair<double, double>> pts, std::vector<double> &hx,
                 std::vector<double> &hy)
{
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    hx.clear();
    hy.clear();
    if (pts.size() < 3) {
        for (auto &p : pts) {
            hx.push_back(p.first);
            hy.push_back(p.second);
        }
        return;
    }
    std::vector<std::pair<double, double>> h(2 * pts.size());
    size_t k = 0;
    for (size_t i = 0; i < pts.size(); ++i) {
        while (k >= 2 && cross(h[k - 2].first, h[k - 2].second, h[k - 1].first, h[k - 1].second,
                               pts[i].first, pts[i].second) <= 0.0)
            --k;
        h[k++] = pts[i];
    }
    for (size_t i = pts.size() - 1, t = k + 1; i-- > 0;) {
        while (k >= t && cross(h[k - 2].first, h[k - 2].second, h[k - 1].first, h[k - 1].second,
                               pts[i].first, pts[i].second) <= 0.0)
            --k;
        h[k++] = pts[i];
    }
    h.resize(k - 1);
    for (auto &p : h) {
        hx.push_back(p.first);
        hy.push_back(p.second);
    }
}

// Area of the intersection of two convex counter-clockwise polygons: clip a
// by every edge of b (Sutherland-Hodgman) and take the shoelace area.
double intersection_area(const Poly &a, const Poly &b)
{
    if (a.x.size() < 3 || b.x.size() < 3)
        return 0.0;
    std::vector<double> px = a.x, py = a.y;
    const size_t nb = b.x.size();
    for (size_t e = 0; e < nb && !px.empty(); ++e) {
        const double ex0 = b.x[e], ey0 = b.y[e];
        const double ex1 = b.x[(e + 1) % nb], ey1 = b.y[(e + 1) % nb];
        std::vector<double> qx, qy;
        const size_t n = px.size();
        for (size_t i = 0; i < n; ++i) {
            const size_t j = (i + 1) % n;
            const double si = cross(ex0, ey0, ex1, ey1, px[i], py[i]);
            const double sj = cross(ex0, ey0, ex1, ey1, px[j], py[j]);
            if (si >= 0.0) {
                qx.push_back(px[i]);
                qy.push_back(py[i]);
            }
            if ((si >= 0.0) != (sj >= 0.0)) {
                const double t = si / (si - sj);
                qx.push_back(px[i] + t * (px[j] - px[i]));
                qy.push_back(py[i] + t * (py[j] - py[i]));
            }
        }
        px.swap(qx);
        py.swap(qy);
    }
    return px.size() < 3 ? 0.0 : std::fabs(shoelace(px, py));
}

}  // namespace

struct pm_map {
    pm_map_params p;
    std::vector<Poly> polys;
    double x = 0.0;   // drift estimate (m)
    double P = 0.0;   // its variance (m^2)
    long long frames = 0;
};

extern "C" {

pm_status pm_map_create(const pm_map_params *p, pm_map **out)
{
    if (!p || !out)
        return pm::set_last_error(PM_ERR_ARG, "null argument");
    *out = nullptr;
    if (!(p->drift_tolerance_m > 0.0) || !(p->sigma_p >= 0.0) || !(p->sigma_m > 0.0) ||
        !(p->initial_variance >= 0.0) || !(p->horizontal_cos > 0.0 && p->horizontal_cos <= 1.0) ||
        !(p->min_overlap_m2 >= 0.0))
        return pm::set_last_error(PM_ERR_ARG, "map parameters out of range");
    pm_map *m = new pm_map;
    m->p = *p;
    m->P = p->initial_variance;
    *out = m;
    return PM_OK;
}

void pm_map_destroy(pm_map *m) { delete m; }

pm_status pm_map_integrate(pm_map *m, const double *pose, const pm_polygon *polys, int n,
                           pm_map_step *step)
{
    if (!m || !pose || (n > 0 && !polys))
        return pm::set_last_error(PM_ERR_ARG, "null argument");
    if (n < 0)
        return pm::set_last_error(PM_ERR_ARG, "negative polygon count");
    for (int i = 0; i < n; ++i)
        if (polys[i].n_vertices < 3 || !polys[i].vertices)
            return pm::set_last_error(PM_ERR_ARG, "a polygon needs at least 3 vertices");
    const double *R = pose;   // row-major 4x4: [R t; 0 1], map <- camera
    // 1. polygons in the map frame: footprint hull, plane, centroid height
    std::vector<Poly> cand;
    int skipped = 0;
    for (int i = 0; i < n; ++i) {
        const pm_polygon &q = polys[i];
        const double nw[3] = {R[0] * q.n[0] + R[1] * q.n[1] + R[2] * q.n[2],
                              R[4] * q.n[0] + R[5] * q.n[1] + R[6] * q.n[2],
                              R[8] * q.n[0] + R[9] * q.n[1] + R[10] * q.n[2]};
        const double nn = std::sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
        if (!(nn > 0.0) || std::fabs(nw[2]) / nn < m->p.horizontal_cos) {
            ++skipped;
            continue;
        }
        // plane n.Xc + d = 0 in the map frame: nw.Xw + dw = 0, dw = d - nw.t
        const double dw = q.d - (nw[0] * R[3] + nw[1] * R[7] + nw[2] * R[11]);
        std::vector<std::pair<double, double>> pts;
        pts.reserve(q.n_vertices);
        for (int k = 0; k < q.n_vertices; ++k) {
            const double *v = q.vertices + 3 * k;
            pts.emplace_back(R[0] * v[0] + R[1] * v[1] + R[2] * v[2] + R[3],
                             R[4] * v[0] + R[5] * v[1] + R[6] * v[2] + R[7]);
        }
        Poly c;
        convex_hull(pts, c.x, c.y);
        c.area = c.x.size() >= 3 ? shoelace(c.x, c.y) : 0.0;
        if (!(c.area > 0.0)) {
            ++skipped;
            continue;
        }
        // area centroid of the footprint, height of the plane there
        double cx = 0.0, cy = 0.0;
        const size_t nv = c.x.size();
        for (size_t a = 0; a < nv; ++a) {
            const size_t b = (a + 1) % nv;
            const double f = c.x[a] * c.y[b] - c.x[b] * c.y[a];
            cx += (c.x[a] + c.x[b]) * f;
            cy += (c.y[a] + c.y[b]) * f;
        }
        cx /= 6.0 * c.area;
        cy /= 6.0 * c.area;
        c.z = -(nw[0] * cx + nw[1] * cy + dw) / nw[2];
        c.observations = 1;
        cand.push_back(std::move(c));
    }
    // 2. matching against the map with the drift estimate of the last frame
    const double tol = m->p.drift_tolerance_m;
    std::vector<int> match(cand.size(), -1);
    double zsum = 0.0;
    int nmatch = 0;
    for (size_t i = 0; i < cand.size(); ++i) {
        double best = tol;
        for (size_t j = 0; j < m->polys.size(); ++j) {
            const double dz = std::fabs(cand[i].z - m->x - m->polys[j].z);
            if (dz <= best && (match[i] < 0 || dz < best) &&
                intersection_area(cand[i], m->polys[j]) > m->p.min_overlap_m2) {
                best = dz;
                match[i] = (int)j;
            }
        }
        if (match[i] >= 0) {
            zsum += cand[i].z - m->polys[match[i]].z;
            ++nmatch;
        }
    }
    // 3. Kalman filter of the vertical drift (Eq. 6-10): one prediction per
    //    frame, an update when the frame matched the map
    const double x_prior = m->x;
    m->P += m->p.sigma_p;
    double K = 0.0, zk = 0.0;
    if (nmatch > 0) {
        zk = zsum / nmatch;
        K = m->P / (m->P + m->p.sigma_m);
        m->x = m->x + K * (zk - m->x);
        m->P = (1.0 - K) * m->P;
    }
    // 4. compensate, merge or add
    int merged = 0, added = 0;
    for (size_t i = 0; i < cand.size(); ++i) {
        Poly &c = cand[i];
        c.z -= m->x;
        if (match[i] < 0) {
            m->polys.push_back(c);
            ++added;
            continue;
        }
        Poly &t = m->polys[match[i]];
        std::vector<std::pair<double, double>> pts;
        for (size_t k = 0; k < t.x.size(); ++k)
            pts.emplace_back(t.x[k], t.y[k]);
        for (size_t k = 0; k < c.x.size(); ++k)
            pts.emplace_back(c.x[k], c.y[k]);
        convex_hull(pts, t.x, t.y);
        t.area = shoelace(t.x, t.y);
        t.observations += 1;
        ++merged;
    }
    m->frames += 1;
    if (step) {
        step->matched = nmatch;
        step->merged = merged;
        step->added = added;
        step->skipped = skipped;
        step->measurement = zk;
        step->gain = K;
        step->drift_prior = x_prior;
        step->drift = m->x;
        step->variance = m->P;
    }
    return PM_OK;
}

int pm_map_size(const pm_map *m) { return m ? (int)m->polys.size() : -1; }

pm_status pm_map_polygon(const pm_map *m, int i, double *height, double *area,
                         int *observations, double *xy, int cap, int *n_vertices)
{
    if (!m || !n_vertices)
        return pm::set_last_error(PM_ERR_ARG, "null argument");
    if (i < 0 || i >= (int)m->polys.size())
        return pm::set_last_error(PM_ERR_ARG, "polygon index out of range");
    const Poly &p = m->polys[i];
    *n_vertices = (int)p.x.size();
    if (height)
        *height = p.z;
    if (area)
        *area = p.area;
    if (observations)
        *observations = p.observations;
    if (xy) {
        const int k = std::min(cap, (int)p.x.size());
        for (int a = 0; a < k; ++a) {
            xy[2 * a] = p.x[a];
            xy[2 * a + 1] = p.y[a];
        }
    }
    return PM_OK;
}

pm_status pm_map_drift(const pm_map *m, double *drift, double *variance)
{
    if (!m)
        return pm::set_last_error(PM_ERR_ARG, "null argument");
    if (drift)
        *drift = m->x;
    if (variance)
        *variance = m->P;
    return PM_OK;
}

}  // extern "C"
